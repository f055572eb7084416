// Batched FP64 eigenvalues of the real-gauge H_eff (row a7: Eq. 1, diagonalising the truncated
// Hamiltonian gives the spectrum E_a of every momentum sector) without a library eigen-solver.
//
// Two kernels per batch of (field, sector) matrices:
//
// 1. sytrd_groups: Householder reduction to tridiagonal form, T = Q^T H Q.  One cooperative
//    launch with two CTAs of 6 warps per SM (one of 12 if two do not fit); the CTAs are shared
//    out among the matrices in proportion to their work (n^3), so a group of C CTAs (1 to 16)
//    owns one matrix and runs all n - 1 reflections, and each SM's two CTAs come from different
//    matrices with even loads (cta_role).  (Hardware thread-block clusters were tried first:
//    their placement left SMs idle, e.g. at most 46 clusters of 3 or 15 of 8 could be resident,
//    so 48 matrices ran in two or more waves.)  Step j builds the reflector v_j from column j,
//    then makes ONE pass over the trailing lower triangle that both applies the rank-2 update
//    of step j - 1,
//        A <- A - v_{j-1} w_{j-1}^T - w_{j-1} v_{j-1}^T,
//    and accumulates the symmetric product y = A v_j for step j; so every trailing element is
//    read and written once per step with four FMAs.  The trailing lower triangle is cut into
//    blocks of 32 rows x 16 columns, and each column group's blocks into chunks of up to
//    kChunk consecutive blocks, with the group's last kTail blocks as a separate tail chunk
//    handed out after all the others.  Warps draw chunks from a per-step ticket counter of the
//    group, so warps and CTAs that run faster (a less busy co-resident CTA, a less crowded
//    SM sub-partition) take more of them.  In a block a lane owns one row: its row sum needs
//    no communication, and its 16 column partial sums stay in registers over the chunk, then
//    one transpose-reduce (16 adds per lane) sums them over the warp.  Two block buffers in
//    registers keep the next block's loads in flight during the current block's arithmetic.
//    Row sums go to a slot per (row, column group) and column sums to a slot per chunk, added
//    in a fixed order, so results do not depend on which warp took which chunk.  The CTAs of
//    a group meet at two barriers per step: an arrival counter in global memory with a
//    bounded wait (a timeout sets an error bit and the kernel returns).  The pass rewrites
//    column j, which the other CTAs read in the same step to build v_j, so a second counter
//    records that each CTA has read it, and a warp waits for it (bounded too) before its
//    first chunk of the group that holds column j.
// 2. sturm_bisect: every eigenvalue by bisection on the Sturm count of T - x, one thread per
//    eigenvalue, with the scaled three-term determinant recurrence (three FP64 operations per
//    row and no divisions; sign changes counted on the integer bits): a grid of counts shared
//    by the block and the first bisection steps in single precision, within a proven error
//    bound; then, for an eigenvalue alone in its bracket, Newton steps on det(T - x) in FP64
//    (kept inside the bracket), else the last bisection steps in FP64.  Persistent blocks draw
//    items of 64 eigenvalues from a queue.
//
// FP64 throughput on this GPU is 1/64 of FP32, so the design counts FP64 instructions: the
// reduction is 4 FMAs per trailing element per step (4n^3/3 flops per matrix); selects, masks,
// sign tests and rescalings are integer operations, and no double value is selected.  The
// matrix is stored in 32 x 16 tiles of 4 KB, so the blocks a warp walks through are sequential
// in memory.
#include <algorithm>
#include <string>
#include <vector>

#include "tgba_internal.h"

namespace tgba {
namespace {

constexpr int kCols = 16;                       // columns of a work block (rows: 32)
constexpr int kMaxGroup = 16;                   // CTAs cooperating on one matrix
constexpr unsigned kSpinLimit = 1u << 24;       // bounded barrier wait (>= 100 ns per poll: over 1 s)
constexpr int kRed = 64;                        // reduction scratch (doubles) after the vectors
constexpr int kChunk = 8;                       // row blocks per chunk of the pass
constexpr int kTail = 2;                        // last blocks of a column group: one chunk, handed out last
constexpr int kMaxSmId = 1024;                  // SM ids registered by cta_role
constexpr int kMaxGroups = kMaxNativeLd / kCols;
constexpr int kSturmThreads = 64;                // bisection block: one item of 64 eigenvalues

struct TriSlot {
  int64_t a_off;    // matrix, ld x ld in 32 x 16 tiles (blk_off), zero beyond n, lower triangle used
  int64_t rp_off;   // row sums of the 32 x 16 blocks [ld][ld / 16]: a row's partials contiguous
  int64_t cp_off;   // column sums of each chunk of a step [chunks][16]
  int64_t tk_off;   // the matrix's step tickets (one counter per step) in the counter array
  int64_t p_off;    // p = tau A v [ld], then one dot partial per CTA of the group [16]
  int64_t de_off;   // diagonal d [n], off-diagonal e [n]
  int64_t out_off;  // first eigenvalue in the caller's output
  int32_t n, ld;
};

__device__ __forceinline__ double isel(bool s, double y, double x) {   // s ? y : x, integer halves
  const int lo = s ? __double2loint(y) : __double2loint(x);
  const int hi = s ? __double2hiint(y) : __double2hiint(x);
  return __hiloint2double(hi, lo);
}

// x if s, else +0.0: the bits ANDed with an all-ones or all-zeros mask (no FP64 instruction)
__device__ __forceinline__ double keep_if(bool s, double x) {
  const int m = s ? -1 : 0;
  return __hiloint2double(__double2hiint(x) & m, __double2loint(x) & m);
}

// Block-tiled storage of an ld x ld matrix: the 32 x 16 block (row block rb, column group g)
// occupies 512 consecutive doubles at ((g LB + rb) 512), column-major inside (column kk of
// the block at + 32 kk), so a warp walking down a column group reads sequential memory.
__device__ __forceinline__ int64_t blk_off(int g, int rb, int LB) { return ((int64_t)g * LB + rb) * (32 * 16); }
__device__ __forceinline__ int64_t elem_off(int i, int k, int LB) {
  return blk_off(k >> 4, i >> 5, LB) + (k & 15) * 32 + (i & 31);
}

// Which CTAs work on which matrix: CTA b takes matrices first, first + stride, ... (each as
// rank `rank` of a group of C CTAs).
struct CtaWork {
  int32_t first, rank, C, stride;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of the C CTAs of one matrix (C = 1: the CTA barrier).  The group's counter counts
// arrivals; the k-th barrier waits until it reaches k C.  Writes before the barrier are
// published by the CTA barrier plus a GPU-scope fence before the arrival, and read after it
// through L2.  The wait is bounded: on timeout it records kStTimeout and returns false, and
// the kernel leaves the matrix (the other CTAs of the group then time out as well).
__device__ __forceinline__ bool group_barrier(unsigned* cnt, unsigned target, int C, int* flag, unsigned* status,
                                              unsigned limit) {
  __syncthreads();
  if (C == 1) return true;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1u);
    int ok = 1;
    for (unsigned it = 0; ld_acquire(cnt) < target; ++it) {
      if (it > limit) {
        ok = 0;
        atomicOr(status, kStTimeout);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// One warp waits (every lane acquiring for itself, bounded like group_barrier) until the
// counter reaches target; on timeout it records kStTimeout and goes on (the result is then
// reported as failed).
__device__ __forceinline__ void warp_wait(const unsigned* cnt, unsigned target, unsigned* status, unsigned limit) {
  for (unsigned it = 0; ld_acquire(cnt) < target; ++it) {
    if (it > limit) {
      if ((threadIdx.x & 31) == 0) atomicOr(status, kStTimeout);
      return;
    }
    __nanosleep(64);
  }
}

// Sum over the block in a fixed order (lane 0 of each warp, then warps in order); every thread
// gets the same value.
template <int WARPS>
__device__ __forceinline__ double block_sum(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double s = red[0];
#pragma unroll
  for (int w = 1; w < WARPS; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Work of one step.  Column group g holds columns 16 g .. 16 g + 15; its blocks are the 32-row
// blocks rb = g / 2 .. LB - 1 (rows 32 rb .. 32 rb + 31, LB = ld / 32), the first on the
// diagonal.  The last min(nb, kTail) blocks of a group form its tail chunk; the blocks before
// it are cut into chunks of up to kChunk.  Chunks 0 .. NCH1 - 1 are those of the heads, group
// by group (cf[t] the first of group g0 + t, cf[NG] = NCH1), and chunk NCH1 + t is group
// g0 + t's tail: so the last chunks of a step are the small ones.
__device__ __forceinline__ int group_head(int g, int LB) { return max(0, LB - (g >> 1) - kTail); }
__device__ __forceinline__ int group_chunks(int g, int LB) { return (group_head(g, LB) + kChunk - 1) / kChunk; }

__device__ __forceinline__ void load_block(double (&a)[kCols], const double* __restrict__ p) {
#pragma unroll
  for (int kk = 0; kk < kCols; ++kk) a[kk] = __ldcg(p + 32 * kk);
}

// One 32 x 16 block held in a[]: row i = 32 rb + lane, columns k0 .. k0 + 15 (p points at the
// lane's element of the block's first column).  vwp[k] = (v_{j-1}, w_{j-1})[k], vwn[k].x =
// v_j[k].  The rank-2 update of the previous step is applied and stored, the row sum of
// A_j v_j over the block's columns goes to rp[i G], the column sums over its rows accumulate in
// cs.  DIAG (the group's first block): elements with row < column add nothing and the
// diagonal element adds only to its row.  Columns left of the trailing block, rows above it
// and padding rows/columns are processed too: there v_{j-1} and w_{j-1} vanish (the update
// leaves the value unchanged, except in column j, which is no longer read), v_j vanishes (no
// row-sum contribution), and the column sums they produce are never read.
template <bool DIAG>
__device__ __forceinline__ void sytrd_block(const double (&a)[kCols], double* __restrict__ p, int i, int k0,
                                            const double2* __restrict__ vwp, const double2* __restrict__ vwn,
                                            double (&cs)[kCols], double* __restrict__ rp, int G) {
  const double2 vwi = vwp[i];
  const double vni = vwn[i].x;
  double r0 = 0.0, r1 = 0.0;
#pragma unroll
  for (int kk = 0; kk < kCols; ++kk) {
    const int k = k0 + kk;
    const double2 vwk = vwp[k];
    const double vnk = vwn[k].x;
    double x = fma(-vwi.x, vwk.y, a[kk]);
    x = fma(-vwi.y, vwk.x, x);
    __stcg(p + 32 * kk, x);
    double& r = (kk & 1) ? r1 : r0;
    if (DIAG) {
      r = fma(x, keep_if(i >= k, vnk), r);
      cs[kk] = fma(x, keep_if(i > k, vni), cs[kk]);
    } else {
      r = fma(x, vnk, r);
      cs[kk] = fma(x, vni, cs[kk]);
    }
  }
  __stcg(rp + (int64_t)i * G, r0 + r1);
}

// Column sums of a warp's run of blocks: cs[m] holds the lane's partial sum of column m.  At
// levels s = 16, 8, 4, 2 a lane keeps half of its values (the upper half if it has bit s set)
// and adds its partner's copy of them, so the values a lane holds halve at every level; a last
// exchange with lane l ^ 1 completes the sum.  Lane l ends with the total of column l >> 1,
// after 16 adds.
__device__ __forceinline__ double transpose_reduce16(double (&cs)[kCols], int lane) {
#pragma unroll
  for (int h = kCols / 2, s = 16; h >= 1; h >>= 1, s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int m = 0; m < h; ++m) {
      const double send = isel(up, cs[m], cs[m + h]);
      const double keep = isel(up, cs[m + h], cs[m]);
      cs[m] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return cs[0] + __shfl_xor_sync(0xffffffffu, cs[0], 1);
}

// Chunk c of the step: row blocks [rb_b, rb_e) of column group g.  Two block buffers in
// registers: the loads of the next block are in flight while the current one is computed.
// The chunk's 16 column sums go to CP[16 c ..].
__device__ __forceinline__ void sytrd_chunk(double* __restrict__ A, int ld, int LB, int g, int rb_b, int rb_e,
                                            int lane, int c, const double2* __restrict__ vwp,
                                            const double2* __restrict__ vwn, double* __restrict__ RP,
                                            double* __restrict__ CP) {
  const int k0 = kCols * g;
  double* gp = A + blk_off(g, 0, LB) + lane;       // + 512 rb: the lane's row of block rb
  double* rp = RP + g;                             // row i's sum at rp[i G]
  const int G = ld / kCols;
  double cs[kCols], cur[kCols], nxt[kCols];
#pragma unroll
  for (int kk = 0; kk < kCols; ++kk) cs[kk] = 0.0;
  int rb = rb_b;
  load_block(cur, gp + 512 * rb);
  if (rb == (g >> 1)) {                            // the diagonal block comes first
    load_block(nxt, gp + 512 * min(rb + 1, rb_e - 1));
    sytrd_block<true>(cur, gp + 512 * rb, 32 * rb + lane, k0, vwp, vwn, cs, rp, G);
    ++rb;
#pragma unroll
    for (int kk = 0; kk < kCols; ++kk) cur[kk] = nxt[kk];
  }
  for (; rb + 1 < rb_e; rb += 2) {
    load_block(nxt, gp + 512 * (rb + 1));
    sytrd_block<false>(cur, gp + 512 * rb, 32 * rb + lane, k0, vwp, vwn, cs, rp, G);
    load_block(cur, gp + 512 * min(rb + 2, rb_e - 1));
    sytrd_block<false>(nxt, gp + 512 * (rb + 1), 32 * (rb + 1) + lane, k0, vwp, vwn, cs, rp, G);
  }
  if (rb < rb_e) sytrd_block<false>(cur, gp + 512 * rb, 32 * rb + lane, k0, vwp, vwn, cs, rp, G);
  const double colsum = transpose_reduce16(cs, lane);
  if ((lane & 1) == 0) __stcg(CP + (int64_t)c * kCols + (lane >> 1), colsum);
}

// All n - 1 reflections of one matrix, as CTA `rank` of its group of C.  Returns false if a
// group barrier gave up.
template <int WARPS>
__device__ __noinline__ bool sytrd_matrix(const TriSlot S, int C, int rank, unsigned* cnt, unsigned* ccnt,
                                          unsigned* tk, double* __restrict__ ws, unsigned* __restrict__ status,
                                          int* flag, unsigned limit) {
  extern __shared__ double sm[];
  unsigned arrivals = 0, col_arrivals = 0;
  const int n = S.n, ld = S.ld, LB = ld >> 5, G = ld / kCols;
  double* A = ws + S.a_off;
  double* RP = ws + S.rp_off;
  double* CP = ws + S.cp_off;
  double* P = ws + S.p_off;
  double* dots = P + ld;
  double* D = ws + S.de_off;
  double* E = D + n;
  double2* vwp = (double2*)sm;                   // (v_{j-1}, w_{j-1}) per index
  double2* vwn = (double2*)(sm + 2 * ld);         // (v_j, w_j)
  double* red = sm + 4 * ld;
  int* cf = (int*)(red + kRed);                   // [NG + 1] first chunk of each group
  __syncthreads();                                // the previous matrix is done with sm
  for (int i = threadIdx.x; i < 4 * ld; i += (WARPS * 32)) sm[i] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool bad = false;
  for (int j = 0; j < n; ++j) {
    // column j of A_j: the stored column (already updated through step j - 2) minus the
    // rank-2 update of step j - 1; rows j + 2 .. n - 1 go into the norm
    const double2 vwj = vwp[j];
    double sig = 0.0;
    for (int i = j + threadIdx.x; i < n; i += (WARPS * 32)) {
      const double2 vwi = vwp[i];
      double a = __ldcg(A + elem_off(i, j, LB));
      a = fma(-vwi.x, vwj.y, a);
      a = fma(-vwi.y, vwj.x, a);
      if (i == j) red[WARPS] = a;
      else if (i == j + 1) red[WARPS + 1] = a;
      else sig = fma(a, a, sig);
      vwn[i].x = a;
    }
    // the step's chunk table (a scan by warp 0 over groups g0 .. G - 1), published by
    // block_sum's barrier
    const int g0 = (j + 1) / kCols, NG = G - g0;
    if (warp == 0) {
      const int per = (NG + 31) >> 5, t0 = min(NG, lane * per), t1 = min(NG, t0 + per);
      int own = 0;
      for (int t = t0; t < t1; ++t) own += group_chunks(g0 + t, LB);
      int incl = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      int run = incl - own;
      for (int t = t0; t < t1; ++t) {
        cf[t] = run;
        run += group_chunks(g0 + t, LB);
      }
      if (lane == 31) cf[NG] = incl;
    }
    sig = block_sum<WARPS>(sig, red);
    // this CTA has read column j (block_sum's barrier): the pass below rewrites it, so the
    // warps that store column j wait until every CTA of the group has arrived here
    if (C > 1 && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(ccnt, 1u);
    }
    col_arrivals += C;
    const double dj = red[WARPS];
    if (rank == 0 && threadIdx.x == 0) D[j] = dj;
    if (j + 1 >= n) break;                            // uniform: the last diagonal entry
    const double alpha = red[WARPS + 1];
    // Householder reflector H = I - tau v v^T with v_{j+1} = 1 mapping column j to beta e_{j+1}
    double beta = alpha, s = 0.0;
    {
      double tau = 0.0;
      if (sig != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, sig));
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        s = 1.0 / (alpha - beta);
      }
      if (threadIdx.x == 0) red[WARPS + 2] = tau;     // read back after the pass
    }
    if (rank == 0 && threadIdx.x == 0) E[j] = beta;
    if (threadIdx.x == 0 && !(isfinite(dj) && isfinite(beta))) bad = true;
    for (int i = threadIdx.x; i < ld; i += (WARPS * 32)) {
      const double x = vwn[i].x;
      vwn[i].x = i == j + 1 ? 1.0 : (i > j + 1 && i < n ? x * s : 0.0);
    }
    __syncthreads();
    // one pass over the trailing lower triangle: update of step j - 1 and y = A_j v_j.  The
    // chunks go out one at a time from the step's ticket counter (the next ticket is drawn
    // while a chunk is computed), so warps and CTAs that run faster take more of them.
    {
      const int NCH1 = cf[NG], NCH = NCH1 + NG;
      bool waited = !(C > 1 && (j + 1) % kCols != 0);   // column j lies in group g0
      unsigned c = 0;
      if (lane == 0) c = atomicAdd(tk + j, 1u);
      c = __shfl_sync(0xffffffffu, c, 0);
      while ((int)c < NCH) {
        unsigned cn = 0;
        if (lane == 0) cn = atomicAdd(tk + j, 1u);
        int lo = 0, rb, re;
        if ((int)c < NCH1) {                          // a head chunk: cf[lo] <= c < cf[lo + 1]
          int hi = NG;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cf[mid] <= (int)c) lo = mid;
            else hi = mid;
          }
          const int gl = g0 + lo;
          rb = (gl >> 1) + ((int)c - cf[lo]) * kChunk;
          re = min(rb + kChunk, (gl >> 1) + group_head(gl, LB));
        } else {                                      // a tail chunk
          lo = (int)c - NCH1;
          const int gl = g0 + lo;
          rb = (gl >> 1) + group_head(gl, LB);
          re = LB;
        }
        const int g = g0 + lo;
        if (lo == 0 && !waited) {
          warp_wait(ccnt, col_arrivals, status, limit);
          waited = true;
        }
        sytrd_chunk(A, ld, LB, g, rb, re, lane, (int)c, vwp, vwn, RP, CP);
        c = __shfl_sync(0xffffffffu, cn, 0);
      }
    }
    arrivals += C;
    if (!group_barrier(cnt, arrivals, C, flag, status, limit)) return false;
    // rows j + 1 .. n - 1, interleaved over the group's CTAs and, within a CTA, over quads of
    // lanes (row i to CTA i mod C; the long rows at the bottom are shared out): y_i = row sums
    // of the blocks of groups g0 .. i/16 + the column sums of the chunks of column i's group.
    // Lane q of the quad adds the partials with index = q mod 4 (four loads in flight each),
    // then the quad adds its four sums in a fixed order; p = tau y
    double dot = 0.0;
    const double tau = red[WARPS + 2];
    {
      const int q4 = lane & 3;
      const int quad = threadIdx.x >> 2, QS = C * (WARPS * 8);      // quads of the group
      const int i_first = j + 1 + rank + C * (threadIdx.x >> 5) * 8;  // the warp's first row
      for (int base = 0; i_first + base < n; base += QS) {
        const int i = j + 1 + rank + C * quad + base;
        double y = 0.0;
        if (i < n) {
          const int gi = i / kCols, t = gi - g0;
          const double* rr = RP + (int64_t)i * G;
          double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
          int g = g0 + q4;
          for (; g + 12 <= gi; g += 16) {
            y0 += __ldcg(rr + g);
            y1 += __ldcg(rr + g + 4);
            y2 += __ldcg(rr + g + 8);
            y3 += __ldcg(rr + g + 12);
          }
          for (; g <= gi; g += 4) y0 += __ldcg(rr + g);
          const int nh = cf[t + 1] - cf[t];             // the group's head chunks, then its tail chunk
          for (int x = q4; x <= nh; x += 4) {
            const int c = x < nh ? cf[t] + x : cf[NG] + t;
            y1 += __ldcg(CP + (int64_t)c * kCols + (i & (kCols - 1)));
          }
          y = (y0 + y1) + (y2 + y3);
        }
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        y += __shfl_xor_sync(0xffffffffu, y, 2);
        if (i < n && q4 == 0) {
          const double p = tau * y;
          __stcg(P + i, p);
          dot = fma(p, vwn[i].x, dot);
        }
      }
    }
    dot = block_sum<WARPS>(dot, red);
    if (threadIdx.x == 0) __stcg(dots + rank, dot);
    arrivals += C;
    if (!group_barrier(cnt, arrivals, C, flag, status, limit)) return false;
    double pv = 0.0;
    for (int r = 0; r < C; ++r) pv += __ldcg(dots + r);
    const double Kc = 0.5 * tau * pv;
    for (int i = threadIdx.x; i < ld; i += (WARPS * 32))
      vwn[i].y = (i > j && i < n) ? fma(-Kc, vwn[i].x, __ldcg(P + i)) : 0.0;
    __syncthreads();
    double2* t = vwp; vwp = vwn; vwn = t;
  }
  if (bad) atomicOr(status, kStEigen);
  return true;
}

// Which CTA plays which role.  A cooperative launch of per_sm CTAs on each of the sms SMs fills
// every SM, but which blockIdx lands on which SM is the hardware's choice, and it can put two
// CTAs of one matrix on one SM (their serial phases then coincide) or two heavy ones together.
// With work_sm given, each CTA registers its SM id (reg[id] counts arrivals per SM, then the
// total and an error flag), and once all have registered takes work_sm[d per_sm + slot], where
// d is the SM's rank among the occupied SM ids and slot its arrival order there; the host
// builds work_sm so that an SM's CTAs come from different matrices and the SMs' loads are even.
// Unless every SM holds exactly per_sm CTAs, all CTAs take work_blk[blockIdx] instead (the
// registration ends the same way for every CTA, so they all decide alike).
__device__ bool cta_role(const CtaWork* __restrict__ work_blk, const CtaWork* __restrict__ work_sm, int per_sm,
                         int sms, unsigned* reg, unsigned* status, CtaWork* out) {
  __shared__ unsigned s_smid, s_slot;
  __shared__ int s_state, s_occ, s_below;
  if (threadIdx.x == 0) {
    s_state = 1;
    s_occ = 0;
    s_below = 0;
    if (work_sm != nullptr) {
      unsigned smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      unsigned slot = 0;
      if (smid < kMaxSmId) slot = atomicAdd(reg + smid, 1u);
      if (smid >= kMaxSmId || slot >= (unsigned)per_sm) atomicOr(reg + kMaxSmId + 1, 1u);
      __threadfence();
      atomicAdd(reg + kMaxSmId, 1u);
      unsigned it = 0;
      while (ld_acquire(reg + kMaxSmId) < gridDim.x && it <= kSpinLimit) {
        __nanosleep(100);
        ++it;
      }
      if (it > kSpinLimit) {
        atomicOr(status, kStTimeout);
        s_state = 0;
      } else {
        s_state = ld_acquire(reg + kMaxSmId + 1) == 0 ? 2 : 1;
      }
      s_smid = smid;
      s_slot = slot;
    }
  }
  __syncthreads();
  const int state = s_state;
  if (state == 0) return false;
  if (state == 2) {
    int occ = 0, below = 0;
    for (int id = threadIdx.x; id < kMaxSmId; id += blockDim.x)
      if (__ldcg(reg + id) != 0u) {
        ++occ;
        below += id < (int)s_smid;
      }
    atomicAdd(&s_occ, occ);
    atomicAdd(&s_below, below);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    *out = (state == 2 && s_occ == sms) ? work_sm[s_below * per_sm + (int)s_slot] : work_blk[blockIdx.x];
  __syncthreads();
  return true;
}

// counters: [B] barrier arrivals, [B] column-j reads, then each matrix's step tickets
// (at 2 B + tk_off, one per step); reg: the SM registration of cta_role.  limit: polls before
// a group wait gives up.  withhold_q >= 0 (failure-detection checks only): the CTA of rank
// withhold_rank in the group of matrix withhold_q leaves after the registration, so the
// group's other CTAs wait for arrivals that never come, until their limit.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 12 / WARPS)
sytrd_groups(const TriSlot* __restrict__ slots, int B, const CtaWork* __restrict__ work_blk,
             const CtaWork* __restrict__ work_sm, int per_sm, int sms, unsigned* __restrict__ reg,
             unsigned* __restrict__ counters, double* __restrict__ ws, unsigned* __restrict__ status,
             unsigned limit, int withhold_q, int withhold_rank) {
  __shared__ int flag;
  __shared__ CtaWork cw_s;
  if (!cta_role(work_blk, work_sm, per_sm, sms, reg, status, &cw_s)) return;
  const CtaWork cw = cw_s;
  const int C = cw.C, rank = cw.rank;
  if (cw.first == withhold_q && rank == withhold_rank) return;
  for (int q = cw.first; q < B; q += cw.stride)
    if (!sytrd_matrix<WARPS>(slots[q], C, rank, counters + q, counters + B + q, counters + 2 * B + slots[q].tk_off,
                             ws, status, &flag, limit))
      return;
}

// Number of eigenvalues of T below x: sign changes of P_0 = 1, P_1, ..., P_n with
// P_{i+1} = (d_i - x) P_i - e_{i-1}^2 P_{i-1}.  A zero P_i is replaced by the smallest normal
// number with the sign opposite to P_{i-1} (the analogue of a negative pivot floor in the ratio
// form), built from integer bits so the FP64 pipe sees only the three operations of the
// recurrence.  Every 8 rows both terms are rescaled by the power of two that brings the larger
// to [1, 2).
__device__ __forceinline__ double nonzero_or_flip(double pn, double pc) {
  const bool z = ((unsigned long long)__double_as_longlong(pn) << 1) == 0ull;
  const int hi = z ? (int)((~(unsigned)__double2hiint(pc) & 0x80000000u) | 0x00100000u) : __double2hiint(pn);
  const int lo = z ? 0 : __double2loint(pn);
  return __hiloint2double(hi, lo);
}

__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double x) {
  double pm = 1.0, pc = nonzero_or_flip(d[0] - x, 1.0);
  int cnt = (int)((unsigned)__double2hiint(pc) >> 31);
  int i = 1;
  for (; i + 8 <= n; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double pn = nonzero_or_flip(fma(d[i + u] - x, pc, -e2[i + u - 1] * pm), pc);
      cnt += (int)((unsigned)(__double2hiint(pn) ^ __double2hiint(pc)) >> 31);
      pm = pc;
      pc = pn;
    }
    const int em = max((__double2hiint(pm) >> 20) & 0x7ff, (__double2hiint(pc) >> 20) & 0x7ff);
    const double sc = __hiloint2double(min(2046, max(1, 2046 - em)) << 20, 0);
    pm *= sc;
    pc *= sc;
  }
  for (; i < n; ++i) {
    const double pn = nonzero_or_flip(fma(d[i] - x, pc, -e2[i - 1] * pm), pc);
    cnt += (int)((unsigned)(__double2hiint(pn) ^ __double2hiint(pc)) >> 31);
    pm = pc;
    pc = pn;
  }
  return cnt;
}

// The characteristic polynomial p(x) = det(T - x) and its derivative by the same three-term
// recurrence, P_{i+1} = (d_i - x) P_i - e_{i-1}^2 P_{i-1} and
// P'_{i+1} = (d_i - x) P'_i - P_i - e_{i-1}^2 P'_{i-1} (five FP64 operations per row; no
// division, so a zero P_i needs no care), all four terms rescaled together every 8 rows.  Only
// the sign of p and the ratio p / p' are used, and the rescaling changes neither.
__device__ __forceinline__ void char_poly(const double* __restrict__ d, const double* __restrict__ e2, int n, double x,
                                          double& p, double& dp) {
  double pm = 1.0, pc = d[0] - x, qm = 0.0, qc = -1.0;
  int i = 1;
  for (; i + 8 <= n; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double t = d[i + u] - x;
      const double pn = fma(t, pc, -e2[i + u - 1] * pm);
      const double qn = fma(t, qc, -fma(e2[i + u - 1], qm, pc));
      pm = pc; pc = pn;
      qm = qc; qc = qn;
    }
    const int em = max(max((__double2hiint(pm) >> 20) & 0x7ff, (__double2hiint(pc) >> 20) & 0x7ff),
                       max((__double2hiint(qm) >> 20) & 0x7ff, (__double2hiint(qc) >> 20) & 0x7ff));
    const double sc = __hiloint2double(min(2046, max(1, 2046 - em)) << 20, 0);
    pm *= sc; pc *= sc;
    qm *= sc; qc *= sc;
  }
  for (; i < n; ++i) {
    const double t = d[i] - x;
    const double pn = fma(t, pc, -e2[i - 1] * pm);
    const double qn = fma(t, qc, -fma(e2[i - 1], qm, pc));
    pm = pc; pc = pn;
    qm = qc; qc = qn;
  }
  p = pc;
  dp = qc;
}

// The same count in single precision on T scaled to norm below 1 (d and e^2 as floats).  It
// is the exact count of a matrix T'(x) with |d'_i - d_i| <= u (2 |d_i| + |x|) and
// |e'_i - e_i| <= 2 u |e_i| (u = 2^-24): the rounding of d - x perturbs d_i, and the roundings
// of e^2 P_{i-2} and of the fused update rescale the terms, which moves into e^2 (the same
// argument as for the ratio form of the recurrence).  So by Weyl's inequality its eigenvalues
// are within 5 u ||T||_inf of T's, and a bracket it finds, widened by 8 u ||T||_inf on each
// side, holds the eigenvalue.  Zero terms take the smallest normal float, as above.
__device__ __forceinline__ float nonzero_or_flip32(float pn, float pc) {
  const unsigned b = __float_as_uint(pn);
  return (b << 1) == 0u ? __uint_as_float((~__float_as_uint(pc) & 0x80000000u) | 0x00800000u) : pn;
}

__device__ __forceinline__ int sturm_count32(const float* __restrict__ d, const float* __restrict__ e2, int n,
                                             float x) {
  float pm = 1.0f, pc = nonzero_or_flip32(d[0] - x, 1.0f);
  int cnt = (int)(__float_as_uint(pc) >> 31);
  int i = 1;
  for (; i + 8 <= n; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float pn = nonzero_or_flip32(fmaf(d[i + u] - x, pc, -e2[i + u - 1] * pm), pc);
      cnt += (int)((__float_as_uint(pn) ^ __float_as_uint(pc)) >> 31);
      pm = pc;
      pc = pn;
    }
    const int em = max((int)((__float_as_uint(pm) >> 23) & 0xff), (int)((__float_as_uint(pc) >> 23) & 0xff));
    const float sc = __uint_as_float((unsigned)min(254, max(1, 254 - em)) << 23);
    pm *= sc;
    pc *= sc;
  }
  for (; i < n; ++i) {
    const float pn = nonzero_or_flip32(fmaf(d[i] - x, pc, -e2[i - 1] * pm), pc);
    cnt += (int)((__float_as_uint(pn) ^ __float_as_uint(pc)) >> 31);
    pm = pc;
    pc = pn;
  }
  return cnt;
}

// Eigenvalues of the tridiagonal matrices by bisection, one thread per eigenvalue (d and e^2 in
// shared memory, as floats for the single-precision steps and then as doubles).  The grid
// is persistent: a block takes items (a matrix and item_len <= 64 consecutive eigenvalue indices) from
// the queue until none is left, so the SMs stay evenly loaded.  Per item: Gershgorin bounds
// [lo, hi] and ||T||; a 64-point grid of single-precision counts shared by the block, then
// single-precision bisection down to a bracket of 2^-21 ||T|| (FP32 runs at 64 times the FP64
// rate on this GPU); the bracket widened by the FP32 count's error bound is checked with two
// FP64 counts (if the check fails the FP64 bisection restarts from the Gershgorin interval),
// then FP64 bisection to 4 eps ||T||, which hands over to Newton's method on det(T - x) as soon
// as the bracket holds the eigenvalue alone (two or three evaluations of five FP64 operations per
// row instead of about 30 counts of three).
__global__ void __launch_bounds__(kSturmThreads)
sturm_bisect(const TriSlot* __restrict__ slots, const int2* __restrict__ items, int n_items, int item_len,
             unsigned* __restrict__ queue, const double* __restrict__ ws, double* __restrict__ evals,
             unsigned* __restrict__ status) {
  extern __shared__ double sm[];
  __shared__ double red[2 * (kSturmThreads / 32)];
  __shared__ int grid_cnt[kSturmThreads];
  __shared__ int item_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    __syncthreads();                                          // the previous item is done with sm
    if (threadIdx.x == 0) item_s = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int it = item_s;
    if (it >= n_items) return;                                // block-uniform
    const int2 wk = items[it];
    const TriSlot S = slots[wk.x];
    const int n = S.n;
    const double* D = ws + S.de_off;
    const double* E = D + n;
    double* d = sm;
    double* e2 = sm + n;
    float* d32 = (float*)sm;                                  // the same memory, first phase
    float* e32 = d32 + n;
    double lo = 1e300, hi = -1e300;
    for (int i = threadIdx.x; i < n; i += kSturmThreads) {
      const double di = D[i];
      const double el = i > 0 ? fabs(E[i - 1]) : 0.0, er = i + 1 < n ? fabs(E[i]) : 0.0;
      lo = fmin(lo, di - el - er);
      hi = fmax(hi, di + el + er);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) { red[warp] = lo; red[kSturmThreads / 32 + warp] = hi; }
    __syncthreads();
    lo = red[0];
    hi = red[kSturmThreads / 32];
    for (int w = 1; w < kSturmThreads / 32; ++w) { lo = fmin(lo, red[w]); hi = fmax(hi, red[kSturmThreads / 32 + w]); }
    const int k = wk.y + threadIdx.x;
    if (!(isfinite(lo) && isfinite(hi))) {                    // block-uniform
      if (threadIdx.x == 0) atomicOr(status, kStEigen);
      if (k < n && (int)threadIdx.x < item_len) evals[S.out_off + k] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const double tnorm = fmax(fabs(lo), fabs(hi));
    // T scaled by a power of two to norm in [0.5, 1): exact in FP64, then rounded to floats
    int ex = 0;
    frexp(tnorm, &ex);
    const double sig = ldexp(1.0, -ex);
    for (int i = threadIdx.x; i < n; i += kSturmThreads) {
      d32[i] = (float)(D[i] * sig);
      e32[i] = i + 1 < n ? (float)(E[i] * E[i] * sig * sig) : 0.0f;
    }
    __syncthreads();
    const double eps = 0x1p-53;
    const double fudge = 4.0 * eps * n * tnorm + 0x1p-1000;  // widen the Gershgorin interval
    const float dl32 = 0x1p-21f * (float)(tnorm * sig);       // 8 u ||T|| (scaled): FP32 count error bound
    // FP32 bracket of the scaled Gershgorin interval, widened by the bound
    const float a0 = __double2float_rd((lo - fudge) * sig) - 2.0f * dl32;
    const float b0 = __double2float_ru((hi + fudge) * sig) + 2.0f * dl32;
    const float step = (b0 - a0) * (1.0f / kSturmThreads);
    if (threadIdx.x > 0) grid_cnt[threadIdx.x] = sturm_count32(d32, e32, n, fmaf(step, (float)threadIdx.x, a0));
    __syncthreads();
    const bool active = k < n && (int)threadIdx.x < item_len;
    float a32 = a0, b32 = b0;                                 // count32(a32) <= k < count32(b32)
    if (active) {
      int c = 1;
      while (c < kSturmThreads && grid_cnt[c] <= k) ++c;      // grid_cnt is non-decreasing in c
      if (c > 1) a32 = fmaf(step, (float)(c - 1), a0);
      if (c < kSturmThreads) b32 = fmaf(step, (float)c, a0);
      for (int i2 = 0; i2 < 64 && b32 - a32 > dl32; ++i2) {
        const float mid = 0.5f * (a32 + b32);
        if (mid <= a32 || mid >= b32) break;
        if (sturm_count32(d32, e32, n, mid) <= k) a32 = mid;
        else b32 = mid;
      }
    }
    __syncthreads();                                          // the FP32 arrays are done with
    for (int i = threadIdx.x; i < n; i += kSturmThreads) {    // d and e^2 in FP64, over them
      d[i] = D[i];
      e2[i] = i + 1 < n ? E[i] * E[i] : 0.0;
    }
    __syncthreads();
    if (!active) continue;
    // FP64: the FP32 bracket widened by the bound, checked; else the Gershgorin interval
    const double dl = (double)dl32 / sig;
    double a = (double)a32 / sig - dl, b = (double)b32 / sig + dl;
    int ca = sturm_count(d, e2, n, a), cb = sturm_count(d, e2, n, b);
    if (!(ca <= k && cb > k)) {
      a = lo - fudge;
      b = hi + fudge;
      ca = 0;
      cb = n;
    }
    const double tol = 4.0 * eps * tnorm + 0x1p-1000;
    // FP64 bisection, keeping the counts of the bracket ends; as soon as the bracket holds
    // this eigenvalue alone (count(a) = k, count(b) = k + 1: at once for most eigenvalues,
    // after a few steps for near-degenerate ones), Newton's method on det(T - x) takes over,
    // kept inside the bracket, which every evaluation narrows (sign(det(T - x)) =
    // (-1)^count(x)); a step that leaves it is replaced by the midpoint.  Converged when a step
    // is below tol; otherwise the bisection finishes from the narrowed bracket.
    bool newton_tried = false;
    for (int i2 = 0; i2 < 200 && b - a > tol; ++i2) {
      if (!newton_tried && ca == k && cb == k + 1) {
        newton_tried = true;
        const bool neg_at_a = (ca & 1) != 0;
        double x = 0.5 * (a + b);
        for (int i3 = 0; i3 < 8 && b - a > tol; ++i3) {
          double pv, dpv;
          char_poly(d, e2, n, x, pv, dpv);
          if (!(isfinite(pv) && isfinite(dpv))) break;
          if (((unsigned)__double2hiint(pv) >> 31) == (neg_at_a ? 1u : 0u)) a = x;
          else b = x;
          if (pv == 0.0) { a = b = x; break; }
          double xn = x - pv / dpv;
          if (fabs(xn - x) <= tol) {                        // converged (the step may touch a bracket end)
            x = fmin(fmax(xn, a), b);
            a = b = x;
            break;
          }
          if (!(xn > a && xn < b)) xn = 0.5 * (a + b);
          x = xn;
        }
        continue;
      }
      const double mid = 0.5 * (a + b);
      if (mid <= a || mid >= b) break;
      const int c = sturm_count(d, e2, n, mid);
      if (c <= k) { a = mid; ca = c; }
      else { b = mid; cb = c; }
    }
    evals[S.out_off + k] = 0.5 * (a + b);
  }
}

// Real-gauge H~ of one (field, sector) slot, full symmetric, ld x ld in 32 x 16 tiles (see
// blk_off); padding rows and columns n .. ld - 1 are zero.  Consecutive threads write
// consecutive doubles of the tiled array.
__global__ void fill_sym(int64_t kn, int64_t kr, int ld, const double* __restrict__ E_ns,
                         const double* __restrict__ E_r, const double* __restrict__ Pm,
                         const double* __restrict__ c0, double scale, double* __restrict__ A) {
  const int64_t n = kn + kr;
  const int LB = ld >> 5;
  const double c = scale * sqrt(c0[0] * c0[0] + c0[1] * c0[1]);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)ld * ld;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = idx >> 9, in = idx & 511;
    const int64_t g = blk / LB, rb = blk - g * LB;
    const int64_t row = rb * 32 + (in & 31), col = g * 16 + (in >> 5);
    double v = 0.0;
    if (row < n && col < n) {
      if (row == col) v = row < kn ? E_ns[row] : E_r[row - kn];
      else if (row < kn && col >= kn) v = c * Pm[row * kr + (col - kn)];
      else if (row >= kn && col < kn) v = c * Pm[col * kr + (row - kn)];
    }
    A[idx] = v;
  }
}

int64_t round32(int64_t x) { return (x + 31) / 32 * 32; }

// Chunks of the first step (g0 = 0), the most of any step.
int64_t max_chunks(int ld) {
  const int LB = ld >> 5;
  int64_t c = 0;
  for (int g = 0; g < ld / kCols; ++g) c += (std::max(0, LB - (g >> 1) - kTail) + kChunk - 1) / kChunk + 1;
  return c;
}

}  // namespace

tgba_status eig_all_sectors_native(Basis& b, const double* hx, int n_hx, double* evals, cudaStream_t st,
                                   const WaitCheck* check) {
  std::vector<TriSlot> slots;
  std::vector<std::pair<int, int>> who;     // (field, sector)
  int64_t total = 0, tk_total = 0;
  int n_max = 0;
  for (int h = 0; h < n_hx; ++h)
    for (size_t s = 0; s < b.sectors.size(); ++s) {
      const int64_t n = b.sectors[s].n_ns + b.sectors[s].n_r;
      if (n == 0) continue;
      TriSlot t{};
      t.n = (int32_t)n;
      t.ld = (int32_t)round32(n);
      t.out_off = (int64_t)h * b.n_states + b.sectors[s].ev_off;
      t.a_off = total;            total += round32((int64_t)t.ld * t.ld);
      t.rp_off = total;           total += round32((int64_t)(t.ld / kCols) * t.ld);
      t.cp_off = total;           total += round32((int64_t)kCols * max_chunks(t.ld));
      t.tk_off = tk_total;        tk_total += t.ld;
      t.p_off = total;            total += round32(t.ld + kMaxGroup);
      t.de_off = total;           total += round32(2 * n);
      slots.push_back(t);
      who.emplace_back(h, (int)s);
      n_max = std::max(n_max, (int)n);
    }
  if (slots.empty()) return TGBA_OK;
  const int B = (int)slots.size();
  int ld_max = 0;
  for (const TriSlot& t : slots) ld_max = std::max(ld_max, t.ld);
  if (ld_max > kMaxNativeLd) return fail(TGBA_EINVAL, "sector too large for the native eigen-solver");
  int dev = 0, sms = 0;
  TGBA_CUDA(cudaGetDevice(&dev));
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // One or two CTAs per SM: two of 6 warps when their shared memory fits (each SM then runs
  // parts of two matrices, and one's barrier waits and serial phases are filled by the other's
  // arithmetic), else one of 12 warps.  With no more matrices than CTAs, every CTA joins one
  // matrix's group: each matrix starts with one CTA and the remaining CTAs go, one at a time,
  // to the matrix with the most work (n^3) per CTA, at most 16 per matrix.  With more matrices
  // than CTAs, CTA b takes matrices b, b + CTAs, ... alone.
  const size_t smem = (size_t)(4 * ld_max + kRed) * sizeof(double) +
                      (size_t)(kMaxGroups + 1) * sizeof(int);
  TGBA_CUDA(cudaFuncSetAttribute(sytrd_groups<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TGBA_CUDA(cudaFuncSetAttribute(sytrd_groups<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TGBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sytrd_groups<6>, 6 * 32, smem));
  per_sm = per_sm >= 2 ? 2 : 1;
  if (per_sm == 1) {
    int one = 0;
    TGBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&one, sytrd_groups<12>, 12 * 32, smem));
    if (one < 1) return fail(TGBA_EINVAL, "the tridiagonalisation's shared memory does not fit on an SM");
  }
  const int ctas = per_sm * sms;
  std::vector<CtaWork> map;
  int C_max = 1;
  if (B <= ctas) {
    std::vector<int> Cq(B, 1);
    for (int left = ctas - B; left > 0; --left) {
      int best = -1;
      double best_w = -1.0;
      for (int q = 0; q < B; ++q) {
        const double w = (double)slots[q].n * slots[q].n * slots[q].n / Cq[q];
        if (Cq[q] < kMaxGroup && w > best_w) { best_w = w; best = q; }
      }
      if (best < 0) break;
      ++Cq[best];
    }
    for (int q = 0; q < B; ++q) {
      for (int r = 0; r < Cq[q]; ++r) map.push_back({q, r, Cq[q], B});
      C_max = std::max(C_max, Cq[q]);
    }
  } else {
    for (int q = 0; q < ctas; ++q) map.push_back({q, 0, 1, ctas});
  }
  const int grid = (int)map.size();
  // The SMs' pairs when every SM holds two CTAs: the CTAs sorted by their work n^3 / C, the
  // k-th heaviest shares an SM with the k-th lightest (even loads), and pairs from one matrix
  // are broken up by exchanging partners with another SM.
  std::vector<CtaWork> sm_map;
  if (per_sm == 2 && grid == ctas) {
    std::vector<int> ord(grid);
    for (int c = 0; c < grid; ++c) ord[c] = c;
    auto wt = [&](int c) { const double n = slots[map[c].first].n; return n * n * n / map[c].C; };
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return wt(x) > wt(y); });
    std::vector<int> lo(sms), hi(sms);
    for (int d = 0; d < sms; ++d) { hi[d] = ord[d]; lo[d] = ord[grid - 1 - d]; }
    for (int d = 0; d < sms; ++d) {
      if (map[hi[d]].first != map[lo[d]].first) continue;
      for (int e = 0; e < sms; ++e)
        if (map[lo[e]].first != map[hi[d]].first && map[hi[e]].first != map[lo[d]].first) {
          std::swap(lo[d], lo[e]);
          break;
        }
    }
    sm_map.resize(grid);
    for (int d = 0; d < sms; ++d) { sm_map[2 * d] = map[hi[d]]; sm_map[2 * d + 1] = map[lo[d]]; }
  }
  const int64_t slot_doubles = round32(((int64_t)B * sizeof(TriSlot) + 7) / 8);
  const int64_t map_doubles = round32(((int64_t)2 * grid * sizeof(CtaWork) + 7) / 8);   // by block, by SM
  // bisection items: item_len consecutive eigenvalue indices of one matrix, 64 (a block's
  // threads) unless that gives fewer items than resident blocks, then 32.  (Items sized to fill
  // whole rounds of the resident blocks, 43 eigenvalues for the 48 L = 24 matrices, measured
  // slower: 25.1 ms against 21.7 ms, the per-item setup outweighing the shorter tail.)
  const size_t smem2 = (size_t)2 * n_max * sizeof(double);   // d, e^2: FP32 first, then FP64, in turn
  TGBA_CUDA(cudaFuncSetAttribute(sturm_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
  int bis_per_sm = 0;
  TGBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bis_per_sm, sturm_bisect, kSturmThreads, smem2));
  if (bis_per_sm < 1) return fail(TGBA_EINVAL, "the bisection's shared memory does not fit on an SM");
  int item_len = kSturmThreads;
  auto count_items = [&](int len) {
    int64_t c = 0;
    for (const TriSlot& t : slots) c += (t.n + len - 1) / len;
    return c;
  };
  if (count_items(item_len) < (int64_t)bis_per_sm * sms) item_len = kSturmThreads / 2;
  std::vector<int2> items;
  for (int q = 0; q < B; ++q)
    for (int k0 = 0; k0 < slots[q].n; k0 += item_len) items.push_back(make_int2(q, k0));
  const int n_items = (int)items.size();
  const int64_t item_doubles = round32(n_items);
  // counters: barriers, column reads, tickets, SM registration, the bisection queue
  const int64_t n_cnt = 2 * (int64_t)B + tk_total + kMaxSmId + 2 + 1;
  const int64_t cnt_doubles = round32((n_cnt + 1) / 2);
  double* ws;
  tgba_status r = scratch(b, total + slot_doubles + map_doubles + cnt_doubles + item_doubles, &ws);
  if (r != TGBA_OK) return r;
  TriSlot* d_slots = (TriSlot*)(ws + total);
  CtaWork* d_map = (CtaWork*)(ws + total + slot_doubles);
  unsigned* d_cnt = (unsigned*)(ws + total + slot_doubles + map_doubles);
  TGBA_CUDA(cudaMemcpyAsync(d_slots, slots.data(), B * sizeof(TriSlot), cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemcpyAsync(d_map, map.data(), grid * sizeof(CtaWork), cudaMemcpyHostToDevice, st));
  CtaWork* d_sm_map = nullptr;
  if (!sm_map.empty()) {
    d_sm_map = d_map + grid;
    TGBA_CUDA(cudaMemcpyAsync(d_sm_map, sm_map.data(), grid * sizeof(CtaWork), cudaMemcpyHostToDevice, st));
  }
  unsigned* d_reg = d_cnt + 2 * B + tk_total;
  unsigned* d_queue = d_reg + kMaxSmId + 2;
  int2* d_items = (int2*)(ws + total + slot_doubles + map_doubles + cnt_doubles);
  TGBA_CUDA(cudaMemcpyAsync(d_items, items.data(), n_items * sizeof(int2), cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemsetAsync(d_cnt, 0, n_cnt * sizeof(unsigned), st));
  for (int q = 0; q < B; ++q) {
    const Sector& sec = b.sectors[who[q].second];
    const int64_t work = (int64_t)slots[q].ld * slots[q].ld;
    const int fgrid = (int)std::min<int64_t>((work + 255) / 256, 152 * 16);
    fill_sym<<<fgrid, 256, 0, st>>>(sec.n_ns, sec.n_r, slots[q].ld, b.d_E_ns + sec.ns_off, b.d_E_r + sec.r_off,
                                    b.d_P + sec.x_off, b.d_c0, -b.L * hx[who[q].first], ws + slots[q].a_off);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(per_sm == 2 ? 6 * 32 : 12 * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident at once: the group barriers rely on it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const unsigned limit = check ? check->spin_limit : kSpinLimit;
  int withhold_q = -1, withhold_rank = -1;
  if (check && check->withhold_matrix >= 0) {
    int C_q = 0;                                 // the group size of that matrix (0: no CTA starts on it)
    for (const CtaWork& w : map)
      if (w.first == check->withhold_matrix) C_q = w.C;
    if (C_q < 2 || check->withhold_rank < 0 || check->withhold_rank >= C_q)
      return fail(TGBA_EINVAL, "the withheld CTA must belong to a group of two or more CTAs");
    withhold_q = check->withhold_matrix;
    withhold_rank = check->withhold_rank;
  }
  for (int e = 0; e < 3; ++e)
    if (b.eig_ev[e] == nullptr) TGBA_CUDA(cudaEventCreate(&b.eig_ev[e]));
  TGBA_CUDA(cudaEventRecord(b.eig_ev[0], st));
  if (per_sm == 2)
    TGBA_CUDA(cudaLaunchKernelEx(&cfg, sytrd_groups<6>, (const TriSlot*)d_slots, B, (const CtaWork*)d_map,
                                 (const CtaWork*)d_sm_map, per_sm, sms, d_reg, d_cnt, ws, b.d_status, limit,
                                 withhold_q, withhold_rank));
  else
    TGBA_CUDA(cudaLaunchKernelEx(&cfg, sytrd_groups<12>, (const TriSlot*)d_slots, B, (const CtaWork*)d_map,
                                 (const CtaWork*)d_sm_map, per_sm, sms, d_reg, d_cnt, ws, b.d_status, limit,
                                 withhold_q, withhold_rank));
  ++b.launches;
  TGBA_CUDA(cudaEventRecord(b.eig_ev[1], st));
  const int bis_grid = std::min(n_items, bis_per_sm * sms);
  sturm_bisect<<<bis_grid, kSturmThreads, smem2, st>>>(d_slots, d_items, n_items, item_len, d_queue, ws, evals,
                                                       b.d_status);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  TGBA_CUDA(cudaEventRecord(b.eig_ev[2], st));
  b.eig_ev_recorded = true;
  double flops = 0;
  for (const TriSlot& t : slots)
    for (int64_t m = 1; m < t.n; ++m) flops += 4.0 * m * (m + 1);
  b.tridiag_flops = flops;
  b.eig_matrices = B;
  b.eig_cluster = C_max;
  return TGBA_OK;
}

}  // namespace tgba
