// FP64 matrix products on the fifth-generation tensor cores, by splitting the FP64 operands
// into BF16 slices (fixed-point digits) whose products the tensor cores sum exactly in FP32.
//
// GB300 runs FP64 at about 1.25 TFLOP/s on its CUDA cores but BF16 MMAs at about 2 PFLOP/s.
// C = A B^T (A: M x K, B: N x K, both with K contiguous in their slices) is computed as follows.
//  * Slicing.  Row i of A gets an exponent e_i with max_k |A_ik| <= 2^e_i; r = A_ik 2^-e_i is
//    cut into S = 6 signed base-256 digits, d_0 = rint(256 r), r <- 256 r - d_0, d_1 = rint(256 r),
//    ... (|d_0| <= 256, |d_p| <= 128 after it; every step exact in FP64), and slice p stores
//    d_p 2^{-8p} in BF16 (exact: at most 8 significant bits).  So A_ik = 2^{e_i - 8} sum_p
//    slice_p + O(2^{e_i - 49}).  B's rows (the columns of C) are cut the same way.
//  * Products.  C_ij = 2^{e_i + f_j - 16} sum_{p + q <= 5} (A_p B_q^T)_ij.  The products of
//    digit diagonal d = p + q carry the scale 2^{-8d}; over a chunk of 256 K values each of
//    the sums of diagonals 0, 1 and 2 stays within 2^24 units of its scale (diagonal 0:
//    256 terms of at most 256 x 256; diagonal 1: 256 x 2 x 256 x 128; diagonal 2 below
//    5 x 2^21), integers that FP32 holds exactly, so FP32 accumulation of those diagonals is
//    exact, and they get one TMEM accumulator each.
//    Diagonals 3..5 share a fourth accumulator, whose FP32 rounding stays near 2^-48 of the
//    leading term (measured: an earlier base-128 split with the shared accumulator from
//    diagonal 3 erred by up to 1.5e-12).
//  * Chunks.  After every 256 K values the four accumulators (4 x 128 columns = all 512 TMEM
//    columns) are folded into a running sum per element kept as an unevaluated pair of FP32
//    numbers (hi + lo, error-free two-sum: about 48 bits), by CUDA-core FP32 arithmetic, while
//    the producer keeps loading the next stages.  At the end of the tile
//    C_ij = 2^{e_i + f_j - 16} (hi + lo) in FP64.
//  The error of C is a few 1e-13 of sum_k |A_ik B_jk| (measured up to 3.9e-13), dominated by
//  the FP32 rounding of the accumulator that the digit diagonals 3..5 share.
//
// Tiles: 128 rows of A x up to 128 rows of B (n_eff, a multiple of 16, per tile) x K in blocks
// of 32 (64-byte rows, 64-byte swizzle).  The slices of one (row block, K block) are stored
// contiguously, already in the shared-memory image the MMA descriptors read, so each stage is
// two bulk copies (cp.async.bulk: 48 KB of A slices, 48 KB of B slices) completing on an
// mbarrier.  Warp 0 issues the copies, warp 1 the MMAs (one thread each), warps 2-9 fold the
// accumulators and write C (each TMEM lane quarter by two warps, 64 columns each).  Two smem
// stages.  N = 128 per MMA instead of 64 halves the shared-memory operand traffic per flop
// (measured at N = 64, the tensor pipe was busy 72% of the active cycles for 31% of its peak
// FLOP rate).  A tile may use fewer columns in later K blocks: per 16-column group the tile
// lists how many K blocks its columns reach, and each block's MMAs take N = the columns still
// active (the first block of a chunk has the most, so it initialises every column the chunk
// folds).
//
// Work split: tiles of 128 x 128 are few (157 for a 20000 x 128 product on 152 SMs: two waves,
// the second nearly empty), so the chunks of all tiles, tile after tile, are cut into one
// contiguous range of equal length per CTA.  A tile cut between CTAs is summed by the last of
// them to finish: each writes its FP64 partial to its slot, bumps a counter per epilogue warp
// (its 32 x 64 block), and the warp that completes the count adds the partials in CTA order
// (no CTA waits for another, and the result does not depend on the arrival order).  Measured:
// 2.06 ms for 20000 x 128 x 20000 against 3.27 ms with whole tiles dealt out in turn, and
// 1.76 ms once the chunks grew from 128 to 256 K values (half as many folds).
//
// Reduced precision: the kernel is also built for the two leading slices only (NS = 2: the
// stages carry 16 KB of each operand, three slice pairs, diagonals 0 and 1), a product good to
// about 2^-16 of the row scales for callers that need only a few digits (spectral bounds).
//
// Every wait is bounded: on
// timeout the kernel records TGBA_ETIMEOUT's status bit, every role leaves, in-flight copies and
// MMAs are waited for (bounded) and the tensor memory is freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <vector>

#include "tgba_internal.h"

namespace tgba {
namespace {

constexpr int kS = 6;                     // slices per operand (base-256 digits)
constexpr int kKB = 32;                   // K per block (64-byte rows)
constexpr int kTMr = 128;                 // rows of A per tile
constexpr int kTNr = 128;                 // rows of B per tile
constexpr int kChunkBlocks = 8;           // K blocks per exact FP32 chunk (256 K values)
constexpr uint32_t kASlice = kTMr * kKB * 2;          // 8 KB
constexpr uint32_t kBSlice = kTNr * kKB * 2;          // 8 KB
constexpr uint32_t kAStage = kS * kASlice;            // 48 KB
constexpr uint32_t kBStage = kS * kBSlice;            // 48 KB
constexpr int kStages = 2;
constexpr uint32_t kSmem = 1024 + kStages * (kAStage + kBStage) + 256;
constexpr unsigned kWait = 1u << 24;                   // polls of a bounded wait
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a tile slice: 64-byte rows, 16-byte chunks XOR (r / 2) mod 4
__host__ __device__ __forceinline__ uint32_t sw64(int r, int k) {
  return (uint32_t)(r * 64 + ((((k >> 3) ^ (r >> 1)) & 3) << 4) + (k & 7) * 2);
}

// Descriptor: start >> 4, LBO 1 (unused for swizzled K-major), SBO 512 B (8-row groups),
// version 1, swizzle mode 4 = 64 B.
__device__ __forceinline__ uint64_t desc64(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)4 << 61);
}

__device__ __forceinline__ uint32_t idesc_f16(int n) {        // D f32, A/B bf16, K-major, M = 128
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTMr >> 4) << 24);
}

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; also gives up when another role has aborted
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag) {
  for (unsigned it = 0; it < kWait; ++it) {
    if (bar_try(b, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// hi + lo += x, error-free (Knuth's two-sum on hi, the error collected in lo)
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}

struct GemmArgs {
  EmuTile* tiles;             // the output tiles, numbered by emu_number_tiles (arrival counters at 0)
  int n_tiles;
  int64_t n_chunks;           // chunks of all tiles (a chunk: kChunkBlocks K blocks of one tile)
  const __nv_bfloat16* A;     // [row block][K block][slice] tile images
  const __nv_bfloat16* B;
  int a_kb, b_kb;             // K blocks per row block of A / of B (the stride between row blocks)
  const int* ea;              // row exponents of A [M]
  const int* eb;              // row exponents of B [N]
  int M, N;
  double* C;                  // C[i + j ldc]
  int64_t ldc;
  double* part;               // [2 gridDim.x][kTNr][kTMr] partial tiles of the split tiles
  unsigned* status;
};

// Work split (stream-K): the chunks of all tiles, tile after tile, are cut into gridDim.x
// contiguous ranges of equal length, one per CTA.  A tile whose chunks fall to several CTAs is
// a split tile: each of them writes its partial sum to a slot of g.part, and the last to arrive
// (an atomic counter in the tile; no CTA waits for another) adds the partials in CTA order and
// writes C, so the result does not depend on the arrival order.
__device__ __forceinline__ int64_t range_start(int c, int64_t T, int G) { return (int64_t)c * T / G; }
__device__ __forceinline__ int cta_of(int64_t x, int64_t T, int G) {    // the CTA whose range holds chunk x
  return (int)(((x + 1) * G + T - 1) / T) - 1;
}
__device__ __forceinline__ int64_t tile_chunks(const EmuTile& t) { return (t.nkb + kChunkBlocks - 1) / kChunkBlocks; }

struct Seg {
  int t;                      // tile
  int kb0, kb1;               // K blocks [kb0, kb1) of the tile
  bool whole;                 // the segment is the whole tile
};
// the segment of tile t from chunk c on (c inside tile t), clipped at the CTA's range end; false past it
__device__ __forceinline__ bool seg_at(const GemmArgs& g, int t, int64_t c, int64_t c_end, Seg& s) {
  if (t >= g.n_tiles || c >= c_end) return false;
  const EmuTile tl = g.tiles[t];
  const int64_t n = tile_chunks(tl), s0 = c - tl.c0, s1 = min(n, c_end - tl.c0);
  s.t = t;
  s.kb0 = (int)(s0 * kChunkBlocks);
  s.kb1 = (int)min((int64_t)tl.nkb, s1 * kChunkBlocks);
  s.whole = s0 == 0 && s1 == n;
  return true;
}
__device__ __forceinline__ int first_tile(const GemmArgs& g, int64_t c) {   // the tile holding chunk c
  int lo = 0, hi = g.n_tiles - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.tiles[mid].c0 <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// columns of the tile that K block kb touches: the 16-column groups whose K extent reaches past it
__device__ __forceinline__ int active_cols(const EmuTile& tl, int kb) {
  int n = 0;
#pragma unroll
  for (int q = 0; q < kTNr / 16; ++q)
    if (q * 16 < tl.n_eff && tl.gkb[q] > kb) n = (q + 1) * 16;
  return n;
}

// NS: slices used per operand, kS (the FP64 product) or 2 (the two leading digits: ~2^-16)
template <int NS>
__global__ void __maxnreg__(168) dgemm_tc_kernel(GemmArgs g) {   // 320 threads x 168 registers, one CTA per SM
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = su32(smem_raw);
  unsigned char* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* sA = base;                                  // [stage] A slices
  unsigned char* sB = base + kStages * kAStage;              // [stage] B slices
  uint64_t* bars = (uint64_t*)(sB + kStages * kBStage);
  uint64_t* full = bars;               // [kStages] stage loaded
  uint64_t* empty = bars + kStages;    // [kStages] stage consumed by the MMAs
  uint64_t* accf = bars + 2 * kStages; // accumulators written (one set)
  uint64_t* acce = accf + 1;           // accumulators read
  uint32_t* tslot = (uint32_t*)(acce + 1);
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(full + s, 1);
      bar_init(empty + s, 1);
    }
    bar_init(accf, 1);
    bar_init(acce, kEpiWarps);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const int G = gridDim.x;
  const int64_t T = g.n_chunks, c_begin = range_start(blockIdx.x, T, G), c_end = range_start(blockIdx.x + 1, T, G);
  const int t_first = first_tile(g, c_begin);

  if (warp == 0) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      Seg sg{t_first - 1, 0, 0, false};
      for (int64_t c = c_begin; !s_abort && seg_at(g, sg.t + 1, c, c_end, sg);
           c = g.tiles[sg.t].c0 + tile_chunks(g.tiles[sg.t])) {
        const EmuTile tl = g.tiles[sg.t];
        for (int kb = sg.kb0; kb < sg.kb1; ++kb, ++it) {
          const int st = it % kStages;
          if (!bar_wait(empty + st, ((it / kStages) & 1u) ^ 1u, &s_abort)) { atomicOr(g.status, kStTimeout); s_abort = 1; break; }
          // the first ns slices of a K block are the first ns x 8 KB of its image
          bar_expect(full + st, (uint32_t)NS * (kASlice + kBSlice));
          bulk_load(sA + st * kAStage, g.A + ((size_t)tl.rb * g.a_kb + kb) * (kAStage / 2), (uint32_t)NS * kASlice,
                    full + st);
          bulk_load(sB + st * kBStage, g.B + ((size_t)tl.cb * g.b_kb + kb) * (kBStage / 2), (uint32_t)NS * kBSlice,
                    full + st);
        }
      }
      if (s_abort) {                                  // copies still in flight land before the CTA leaves
        const volatile int never = 0;
        for (uint32_t j = (it >= kStages ? it - kStages : 0); j < it; ++j)
          bar_wait(full + (j % kStages), (j / kStages) & 1u, (volatile int*)&never);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t it = 0, chunk = 0;
      uint64_t* last = nullptr;
      Seg sg{t_first - 1, 0, 0, false};
      for (int64_t c = c_begin; !s_abort && seg_at(g, sg.t + 1, c, c_end, sg);
           c = g.tiles[sg.t].c0 + tile_chunks(g.tiles[sg.t])) {
        const EmuTile tl = g.tiles[sg.t];
        for (int kb0 = sg.kb0; kb0 < sg.kb1 && !s_abort; kb0 += kChunkBlocks, ++chunk) {
          // the epilogue has read the previous chunk's accumulators
          if (!bar_wait(acce, (chunk & 1u) ^ 1u, &s_abort)) { atomicOr(g.status, kStTimeout); s_abort = 1; break; }
          fence_after();
          const int kb1 = min(sg.kb1, kb0 + kChunkBlocks);
          for (int kb = kb0; kb < kb1; ++kb, ++it) {
            const int st = it % kStages;
            if (!bar_wait(full + st, (it / kStages) & 1u, &s_abort)) { atomicOr(g.status, kStTimeout); s_abort = 1; break; }
            fence_after();
            // columns whose K extent ends before this block are skipped (their rows of B are zero
            // there); the chunk's first block touches the most columns, so its MMAs initialise
            // every column that the epilogue reads
            const uint32_t id = idesc_f16(active_cols(tl, kb));
            const uint32_t a0 = su32(sA + st * kAStage), b0 = su32(sB + st * kBStage);
#pragma unroll 1
            for (int p = 0; p < NS; ++p)
#pragma unroll 1
              for (int q = 0; p + q < NS; ++q) {
                const int d = min(p + q, 3);
                // first write of accumulator d in this chunk overwrites it: pair (0, d) for d <= 2,
                // (0, 3) for the shared one, at the chunk's first K block
                const bool first = kb == kb0 && p == 0 && q == (d < 3 ? d : 3);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                  mma(tmem + (uint32_t)d * 128u, desc64(a0 + p * kASlice + ks * 32), desc64(b0 + q * kBSlice + ks * 32), id,
                      (first && ks == 0) ? 0u : 1u);
              }
            commit(empty + st);                       // the stage's smem is free once these complete
            last = empty + st;
          }
          commit(accf);                               // the chunk's accumulators are complete
          last = accf;
        }
      }
      if (s_abort && last) {                          // MMAs still in flight finish before the dealloc
        const volatile int never = 0;
        bar_wait(last, 0u, (volatile int*)&never);
        bar_wait(last, 1u, (volatile int*)&never);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue (warps 2-9)
    constexpr int kCols = kTNr / 2;                   // columns per epilogue warp
    const int quad = warp & 3;                        // TMEM lanes 32 quad .. 32 quad + 31
    const int half = (warp - 2) >> 2;                 // columns kCols half .. kCols half + kCols - 1
    const int r = quad * 32 + lane;                   // row of the tile
    uint32_t chunk = 0;
    Seg sg{t_first - 1, 0, 0, false};
    for (int64_t c = c_begin; !s_abort && seg_at(g, sg.t + 1, c, c_end, sg);
         c = g.tiles[sg.t].c0 + tile_chunks(g.tiles[sg.t])) {
      const EmuTile tl = g.tiles[sg.t];
      float hi[kCols], lo[kCols];                     // registers: every index below is a constant
#pragma unroll
      for (int cc = 0; cc < kCols; ++cc) { hi[cc] = 0.f; lo[cc] = 0.f; }
      for (int kb0 = sg.kb0; kb0 < sg.kb1; kb0 += kChunkBlocks, ++chunk) {
        if (!bar_wait(accf, chunk & 1u, &s_abort)) {
          if (lane == 0) atomicOr(g.status, kStTimeout);
          s_abort = 1;
          break;
        }
        fence_after();
        const int na = active_cols(tl, kb0);          // columns the chunk's MMAs wrote
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * kCols);
#pragma unroll
        for (int h = 0; h < kCols / 16; ++h) {
          if (half * kCols + h * 16 < na) {
#pragma unroll
            for (int d = 0; d < (NS < 4 ? NS : 4); ++d) {   // with 2 slices only diagonals 0 and 1 are written
              float v[16];
              ld16(lane_base + (uint32_t)d * (uint32_t)kTNr + (uint32_t)h * 16u, v);
#pragma unroll
              for (int j = 0; j < 16; ++j) two_sum_add(hi[h * 16 + j], lo[h * 16 + j], v[j]);
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(acce);
      }
      if (s_abort) break;
      const int i = tl.rb * kTMr + r;
      const int c_lo = half * kCols;
      if (sg.whole) {
        if (i < g.M) {
          const int e_i = g.ea[i];
#pragma unroll
          for (int cc = 0; cc < kCols; ++cc) {
            const int j = tl.cb * kTNr + c_lo + cc;
            if (c_lo + cc < tl.n_eff && j < g.N)
              g.C[(int64_t)i + (int64_t)j * g.ldc] = ldexp((double)hi[cc] + (double)lo[cc], e_i + g.eb[j] - 16);
          }
        }
        continue;
      }
      // split tile: this CTA's partial to its slot (0: the tile its range starts in, 1: the tile it ends in)
      const int slot = 2 * (int)blockIdx.x + (sg.t == t_first ? 0 : 1);
      double* mine = g.part + (size_t)slot * kTNr * kTMr;
#pragma unroll
      for (int cc = 0; cc < kCols; ++cc)
        if (c_lo + cc < tl.n_eff) mine[(size_t)(c_lo + cc) * kTMr + r] = (double)hi[cc] + (double)lo[cc];
      // the last of the tile's CTAs to finish this warp's 32 x 64 block adds the parts (no waiting)
      __threadfence();
      __syncwarp();
      const int c_a = cta_of(tl.c0, T, G), c_b = cta_of(tl.c0 + tile_chunks(tl) - 1, T, G);
      int last = 0;
      if (lane == 0) last = atomicAdd(&g.tiles[sg.t].arrivals[warp - 2], 1) == c_b - c_a;
      if (__shfl_sync(0xffffffffu, last, 0)) {
        __threadfence();
        if (i < g.M) {
          const int e_i = g.ea[i];
#pragma unroll 4
          for (int cc = 0; cc < kCols; ++cc) {
            const int j = tl.cb * kTNr + c_lo + cc;
            if (c_lo + cc < tl.n_eff && j < g.N) {
              double v = 0.0;
              for (int cta = c_a; cta <= c_b; ++cta) {
                const int sl = 2 * cta + (range_start(cta, T, G) >= tl.c0 ? 0 : 1);
                v += __ldcg(g.part + (size_t)sl * kTNr * kTMr + (size_t)(c_lo + cc) * kTMr + r);
              }
              g.C[(int64_t)i + (int64_t)j * g.ldc] = ldexp(v, e_i + g.eb[j] - 16);
            }
          }
        }
        if (lane == 0) g.tiles[sg.t].arrivals[warp - 2] = 0;   // every part has arrived: ready for the next launch
      }
    }
  }
  // teardown: everything issued has completed or been abandoned after a bounded wait
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// GB300's FP64 pipe is slow, so the slicing works on the bit patterns with integer operations
// (only the optional weight takes two FP64 operations per element).
__device__ __forceinline__ double weighted(const double* __restrict__ src, int64_t off, const double* __restrict__ w,
                                          double w_shift, int k) {
  const double x = src[off];
  return w ? x * (w[k] - w_shift) : x;
}

// Row exponents: e[i] = smallest e with max_k |X(i, k)| < 2^e (0 for a zero row), from the
// largest magnitude's exponent field (integer maximum of the magnitudes' bit patterns).  One
// warp per row.
__global__ void row_exponents(int rows, int K, const double* __restrict__ src, int64_t row_stride, int64_t k_stride,
                              int k_split, int64_t k_jump, const double* __restrict__ w, double w_shift,
                              int* __restrict__ e) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += (gridDim.x * blockDim.x) >> 5) {
    unsigned long long m = 0ull;
    for (int k = lane; k < K; k += 32) {
      const int64_t off = (int64_t)i * row_stride + (int64_t)k * k_stride + (k >= k_split ? k_jump : 0);
      unsigned long long bits;                           // magnitude bits (an integer AND, not fabs)
      asm("and.b64 %0, %1, 0x7fffffffffffffff;"
          : "=l"(bits)
          : "l"((unsigned long long)__double_as_longlong(weighted(src, off, w, w_shift, k))));
      m = max(m, bits);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      const int ef = (int)(m >> 52);                     // biased exponent of the largest magnitude
      e[i] = m == 0ull ? 0 : (ef == 0 ? -1021 : ef - 1022);   // max < 2^(ef - 1022)
    }
  }
}

// The same with one block of 256 threads per row, for few long rows (the vectors of the
// Chebyshev steps: 128 rows of up to 4e4): a warp per row would leave most SMs idle.
__global__ void row_exponents_long(int rows, int K, const double* __restrict__ src, int64_t row_stride,
                                   int64_t k_stride, int k_split, int64_t k_jump, const double* __restrict__ w,
                                   double w_shift, int* __restrict__ e) {
  __shared__ unsigned long long s_m[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < rows; i += gridDim.x) {
    unsigned long long m = 0ull;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const int64_t off = (int64_t)i * row_stride + (int64_t)k * k_stride + (k >= k_split ? k_jump : 0);
      unsigned long long bits;
      asm("and.b64 %0, %1, 0x7fffffffffffffff;"
          : "=l"(bits)
          : "l"((unsigned long long)__double_as_longlong(weighted(src, off, w, w_shift, k))));
      m = max(m, bits);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_m[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = max(m, s_m[q]);
      const int ef = (int)(m >> 52);
      e[i] = m == 0ull ? 0 : (ef == 0 ? -1021 : ef - 1022);
    }
    __syncthreads();
  }
}

// Slices of X (rows x K, element (i, k) at src[i row_stride + k k_stride (+ k_jump for k >= k_split)],
// optionally times w[k] - w_shift) as tile images [row block][K block][slice][tile rows][32] (bf16,
// 64-byte swizzle); rows and K beyond the matrix are zero.  The value 2^-e x (|.| < 1) is rounded
// to a 48-bit fixed-point integer F (from the mantissa and exponent fields), which is cut into
// six balanced base-256 digits, d_p = round(F / 2^(40 - 8p)), F -= d_p 2^(40 - 8p).
__global__ void slice_tiles(int rows, int K, const double* __restrict__ src, int64_t row_stride, int64_t k_stride,
                            int k_split, int64_t k_jump, const double* __restrict__ w, double w_shift,
                            const int* __restrict__ e, int tile_rows, int n_kb, __nv_bfloat16* __restrict__ out) {
  // one thread per 8 consecutive K values of a row: each slice gets one 16-byte store (the
  // 64-byte swizzle moves whole 16-byte chunks, so the 8 values stay contiguous)
  const int n_rb = (rows + tile_rows - 1) / tile_rows;
  const int64_t k8s = (int64_t)n_kb * (kKB / 8);
  const int64_t total = (int64_t)n_rb * tile_rows * k8s;
  const uint32_t slice_bytes = (uint32_t)tile_rows * kKB * 2;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int k8 = (int)(q % k8s);
    const int i = (int)(q / k8s);
    const int k0 = k8 * 8;
    const int rb = i / tile_rows, r = i % tile_rows, kb = k0 / kKB, kk = k0 % kKB;
    long long F[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u;
      F[u] = 0;
      if (i < rows && k < K) {
        const int64_t off = (int64_t)i * row_stride + (int64_t)k * k_stride + (k >= k_split ? k_jump : 0);
        const unsigned long long bits = (unsigned long long)__double_as_longlong(weighted(src, off, w, w_shift, k));
        const int ef = (int)((bits >> 52) & 0x7ff);
        if (ef != 0) {                                   // subnormals are below 2^-1022: they round to 0
          const long long mant = (long long)((bits & 0x000fffffffffffffull) | 0x0010000000000000ull);
          // |x| = mant 2^(ef - 1075); F = |x| 2^(48 - e) = mant 2^(ef - 1027 - e), a right shift
          const int sh = 1027 + e[i] - ef;
          long long f = 0;
          if (sh <= 0) f = mant << (-sh);                // only for |x| at the top of the range
          else if (sh < 63) f = (mant + (1ll << (sh - 1))) >> sh;
          F[u] = (bits >> 63) ? -f : f;
        }
      }
    }
    unsigned char* tile = (unsigned char*)out + ((size_t)rb * n_kb + kb) * kS * slice_bytes + sw64(r, kk);
#pragma unroll
    for (int p = 0; p < kS; ++p) {
      const int shp = 40 - 8 * p;
      uint32_t packed[4];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long d = shp > 0 ? ((F[u] + (1ll << (shp - 1))) >> shp) : F[u];
        F[u] -= d << shp;
        // d 2^(-8p): |d| <= 256, exact in FP32 and in BF16
        const uint32_t h = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(ldexpf((float)d, -8 * p)));
        if (u & 1) packed[u >> 1] |= h << 16;
        else packed[u >> 1] = h;
      }
      *(uint4*)(tile + (size_t)p * slice_bytes) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
  }
}

}  // namespace

size_t emu_operand_elems(int rows, int K, int tile_rows) {
  const int n_rb = (rows + tile_rows - 1) / tile_rows, n_kb = (K + kKB - 1) / kKB;
  return (size_t)n_rb * n_kb * kS * tile_rows * kKB;
}

// Slices of a matrix X (rows x K) for dgemm_tc: element (i, k) at src[i row_stride + k k_stride],
// k >= k_split shifted by k_jump more (two K ranges of one buffer); if w != nullptr, times
// (w[k] - w_shift).  out: bf16 [emu_operand_elems], e: int [rows].  tile_rows: 128 for A, 64 for B.
tgba_status emu_slice(Basis& b, const double* src, int64_t row_stride, int64_t k_stride, int k_split, int64_t k_jump,
                      const double* w, double w_shift, int rows, int K, int tile_rows, __nv_bfloat16* out, int* e,
                      cudaStream_t st) {
  if (rows <= 0 || K <= 0) return TGBA_OK;
  const int n_kb = (K + kKB - 1) / kKB;
  if (rows < 152 * 8 && K >= 1024)
    row_exponents_long<<<rows, 256, 0, st>>>(rows, K, src, row_stride, k_stride, k_split, k_jump, w, w_shift, e);
  else
    row_exponents<<<(int)std::min<int64_t>(((int64_t)rows * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
        rows, K, src, row_stride, k_stride, k_split, k_jump, w, w_shift, e);
  ++b.launches;
  const int n_rb = (rows + tile_rows - 1) / tile_rows;
  const int64_t total = (int64_t)n_rb * tile_rows * n_kb * (kKB / 8);
  slice_tiles<<<(int)std::min<int64_t>((total + 255) / 256, 152 * 64), 256, 0, st>>>(
      rows, K, src, row_stride, k_stride, k_split, k_jump, w, w_shift, e, tile_rows, n_kb, out);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

// Kernel attributes and the SM count, once per device (outside any stream capture); the
// partial-tile workspace of the work split, once per handle.
tgba_status emu_prepare(Basis& b) {
  static int sms_of[64] = {0};
  if (b.device < 0 || b.device >= 64) return fail(TGBA_ELIMIT, "device index");
  if (sms_of[b.device] == 0) {
    for (const void* k : {(const void*)dgemm_tc_kernel<kS>, (const void*)dgemm_tc_kernel<2>}) {
      TGBA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
      cudaFuncAttributes fa;
      TGBA_CUDA(cudaFuncGetAttributes(&fa, k));
      if (fa.maxThreadsPerBlock < kThreads) {
        char msg[200];
        snprintf(msg, sizeof msg, "dgemm_tc_kernel: %d registers, %zu B local, %zu B static shared: at most %d threads",
                 fa.numRegs, fa.localSizeBytes, fa.sharedSizeBytes, fa.maxThreadsPerBlock);
        return fail(TGBA_ELIMIT, msg);
      }
    }
    int sms = 0;
    TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
    sms_of[b.device] = sms;
  }
  b.emu_sms = sms_of[b.device];
  if (!b.d_emu_part) TGBA_CUDA(cudaMalloc(&b.d_emu_part, emu_part_bytes(b.emu_sms)));
  return TGBA_OK;
}

size_t emu_part_bytes(int sms) { return (size_t)2 * sms * kTNr * kTMr * sizeof(double); }

int64_t emu_number_tiles(std::vector<EmuTile>& tiles) {
  int64_t c = 0;
  for (EmuTile& t : tiles) {
    if (t.nkb < 1 || t.n_eff < 16 || t.n_eff > kTNr || t.n_eff % 16) return -1;
    t.c0 = c;
    for (int q = 0; q < kTNr / 16; ++q) {
      t.arrivals[q] = 0;
      if (t.gkb[q] <= 0 || t.gkb[q] > t.nkb) t.gkb[q] = (int16_t)t.nkb;   // unset: the tile's whole K
    }
    c += (t.nkb + kChunkBlocks - 1) / kChunkBlocks;
  }
  return c;
}

// C = A B^T for sliced operands (see emu_slice), over the given output tiles (numbered by
// emu_number_tiles, n_chunks its result; emu_prepare first).
tgba_status emu_gemm(Basis& b, const __nv_bfloat16* A, const int* ea, int M, int Ka, const __nv_bfloat16* B,
                     const int* eb, int N, int Kb, EmuTile* d_tiles, int n_tiles, int64_t n_chunks, double* C,
                     int64_t ldc, cudaStream_t st, int n_slices) {
  if (n_slices != 2 && n_slices != kS) return fail(TGBA_EINVAL, "emu_gemm: 2 or 6 slices");
  if (n_tiles == 0) return TGBA_OK;
  if (b.emu_sms <= 0 || !b.d_emu_part) return fail(TGBA_EINVAL, "emu_prepare was not called");
  if (n_chunks < n_tiles) return fail(TGBA_EINVAL, "tiles not numbered (emu_number_tiles)");
  GemmArgs g;
  g.tiles = d_tiles; g.n_tiles = n_tiles; g.n_chunks = n_chunks;
  g.A = A; g.B = B;
  g.a_kb = (Ka + kKB - 1) / kKB;
  g.b_kb = (Kb + kKB - 1) / kKB;
  g.ea = ea; g.eb = eb; g.M = M; g.N = N; g.C = C; g.ldc = ldc; g.part = b.d_emu_part; g.status = b.d_status;
  const int grid = (int)std::min<int64_t>(n_chunks, b.emu_sms);
  if (n_slices == kS) dgemm_tc_kernel<kS><<<grid, kThreads, kSmem, st>>>(g);
  else dgemm_tc_kernel<2><<<grid, kThreads, kSmem, st>>>(g);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

int emu_tile_rows_a() { return kTMr; }
int emu_tile_rows_b() { return kTNr; }
int emu_k_block() { return kKB; }

}  // namespace tgba

extern "C" tgba_status tgba_dgemm_tc(int32_t M, int32_t N, int32_t K, const double* A, int64_t lda, const double* B,
                                     int64_t ldb, double* C, int64_t ldc, void* stream) {
  using namespace tgba;
  if (M < 1 || N < 1 || K < 1) return fail(TGBA_EINVAL, "need M, N, K >= 1");
  if (!A || !B || !C) return fail(TGBA_EINVAL, "null pointer");
  if (lda < K || ldb < K || ldc < M) return fail(TGBA_EINVAL, "leading dimensions too small");
  cudaStream_t st = (cudaStream_t)stream;
  Basis ctx;
  TGBA_CUDA(cudaGetDevice(&ctx.device));
  const size_t ea = emu_operand_elems(M, K, emu_tile_rows_a()), eb = emu_operand_elems(N, K, emu_tile_rows_b());
  const int TR = emu_tile_rows_a(), TC = emu_tile_rows_b(), KB = emu_k_block();
  std::vector<EmuTile> tiles;
  for (int rb = 0; rb < (M + TR - 1) / TR; ++rb)
    for (int cb = 0; cb < (N + TC - 1) / TC; ++cb)
      tiles.push_back(EmuTile{rb, cb, std::min(TC, (N - cb * TC + 15) / 16 * 16), (K + KB - 1) / KB});
  const int64_t n_chunks = emu_number_tiles(tiles);
  if (n_chunks < 0) return fail(TGBA_EINVAL, "tile list");
  int sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx.device));
  void* buf = nullptr;
  const size_t bytes = emu_part_bytes(sms) + (ea + eb) * 2 + (size_t)(M + N) * 4 + tiles.size() * sizeof(EmuTile) + 64;
  cudaError_t e = cudaMallocAsync(&buf, bytes, st);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(TGBA_ENOMEM, "slice buffers of tgba_dgemm_tc"); }
  struct Free { void* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{buf, st};
  ctx.d_emu_part = (double*)buf;                      // the handle-less call brings its own workspace
  __nv_bfloat16* As = (__nv_bfloat16*)((char*)buf + emu_part_bytes(sms));
  __nv_bfloat16* Bs = As + ea;
  int* xa = (int*)(Bs + eb);
  int* xb = xa + M;
  EmuTile* dt = (EmuTile*)(((uintptr_t)(xb + N) + 15) & ~(uintptr_t)15);
  ctx.d_status = (unsigned*)(dt + tiles.size());
  TGBA_CUDA(cudaMemsetAsync(ctx.d_status, 0, sizeof(unsigned), st));
  TGBA_CUDA(cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
  tgba_status r = emu_prepare(ctx);
  if (r == TGBA_OK) r = emu_slice(ctx, A, lda, 1, K, 0, nullptr, 0.0, M, K, TR, As, xa, st);
  if (r == TGBA_OK) r = emu_slice(ctx, B, ldb, 1, K, 0, nullptr, 0.0, N, K, TC, Bs, xb, st);
  if (r == TGBA_OK) r = emu_gemm(ctx, As, xa, M, K, Bs, xb, N, K, dt, (int)tiles.size(), n_chunks, C, ldc, st);
  if (r != TGBA_OK) return r;
  unsigned w = 0;
  TGBA_CUDA(cudaMemcpyAsync(&w, ctx.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  ctx.d_status = nullptr;
  ctx.d_emu_part = nullptr;
  if (w & kStTimeout) return fail(TGBA_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up");
  return TGBA_OK;
}
