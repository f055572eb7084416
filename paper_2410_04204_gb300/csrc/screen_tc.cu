// Screener inference on the fifth-generation tensor cores (row a5): layer 2 of the pair MLP as
// tcgen05 MMAs with the accumulator in tensor memory, fused with layer 1, layer 3, the
// threshold and the compaction of the kept pairs into per-size work lists.
//
// A pair (a, b) has h1 = relu(A_a + B_b) (the per-state layer-1 partials, FP32), z2 = W2 h1 + b2,
// y = w3 . relu(z2) + b3.  One persistent CTA per SM holds W2 (BF16, 256 x 256, 128 KB) in
// shared memory for the whole launch.  Per tile of 8 x 16 pairs (8 NS states by 16 R states)
// of one rectangle of uniform (M_a, M_b) (hence uniform Pfaffian size n):
//   0. the CTA loads the tile's 8 + 16 partial rows (24 KB, coalesced) into shared memory, once
//      per tile instead of once per pair (a tile of 128 pairs along one row read 128 R rows
//      and one NS row, 129 KB, through L1);
//   1. each of the 128 threads builds its pair's row of h1 (BF16) in shared memory, in the
//      K-major layout with the 128-byte swizzle that the MMA's shared-memory descriptors read;
//   2. one thread issues 16 MMAs (M = 128, N = 256, K = 16 each: D[128 x 256] += A B^T) into a
//      256-column FP32 accumulator in tensor memory, then commits them to an mbarrier;
//   3. after the barrier each warp loads its 32 rows of the accumulator (tcgen05.ld) and forms
//      y = w3 . relu(z2 + b2) + b3 per row;
//   4. a pair is kept when y - (n/2) log10(L/24) + log10(L |h_x|) >= log10(tau) - margin, or when
//      a state has more quasiparticles than the model's features hold; kept pairs go to the
//      work list of their size (one atomic per tile), and (prediction mode) y is stored.
// Every mbarrier wait is bounded: on timeout the kernel records TGBA_ETIMEOUT's status bit,
// waits (bounded again) for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "tgba_internal.h"

namespace tgba {
namespace {

constexpr int kH = 256;                 // MLP width (N and K of the layer-2 MMA)
constexpr int kTM = 128;                // pairs per tile (M of the MMA)
constexpr int kTR = 8, kTC = 16;        // the tile's NS states x R states
constexpr int kPartStride = kH + 4;     // floats per staged partial row (16 B of padding: the 16
                                        // R rows a warp reads start in different banks)
constexpr int kModelQp = 8;             // quasiparticles the features hold per state
constexpr uint32_t kBBytes = kH * kH * 2;             // W2 in BF16: 128 KB
constexpr uint32_t kABytes = kTM * kH * 2;            // one h1 tile: 64 KB
constexpr uint32_t kPartBytes = (kTR + kTC) * kPartStride * 4;   // staged partials: 24.4 KB
constexpr uint32_t kSmemBytes = 1024 + kBBytes + kABytes + 2 * kH * 4 + 64 + kPartBytes;
constexpr unsigned kWaitLimit = 1u << 22;             // polls of a bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-dimension offset >> 4
// (bits 16-29; not used by K-major swizzled layouts, set to 1), stride-dimension offset >> 4
// (bits 32-45: 1024 B between groups of 8 rows), version 1 (bit 46), swizzle mode 2 = 128 B
// (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// Byte offset of element (row, k) of a K-major BF16 tile with `rows` rows, K = 256: four column
// blocks of 64 elements (128 B per row); inside a block, 8-row groups of 1024 B and the 16-byte
// chunks of a row permuted by XOR with (row mod 8) (the 128-byte swizzle).
__device__ __forceinline__ uint32_t swz(int rows, int row, int chunk16) {   // chunk16: 0..31 along K
  const int kc = chunk16 >> 3, c = chunk16 & 7;
  return (uint32_t)(kc * rows * 128 + row * 128 + ((c ^ (row & 7)) << 4));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase with parity `phase` to complete; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned phase) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

struct ScoreArgs {
  const Rect* rects;          // rectangles of uniform (M_a, M_b)
  const int64_t* prefix;      // [n_rects + 1] first 8 x 16 tile of each rectangle
  int n_rects;
  int64_t n_tiles;
  const float* Apart;         // per NS state (global index): A_a [kH]
  const float* Bpart;         // per R state: B_b (b1 included) [kH]
  const __nv_bfloat16* W2b;   // [kH][kH], row = output unit
  const float* b2;
  const float* w3;
  const float* b3;
  float shift, half_log_l;
  float* pred;                // optional: y at (out index - pred_base)
  int64_t pred_base;
  unsigned* counts;           // optional list mode: kept pairs per size n / 2
  const int64_t* list_off;    // first entry of each size's list
  PairEntry* lists;
  unsigned* status;
};

__device__ __forceinline__ int tile_rect(const int64_t* __restrict__ prefix, int n, int64_t t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kTM, 1) score_tc(ScoreArgs g) {
  extern __shared__ unsigned char smem_raw[];
  // swizzle atoms need 1024-byte aligned shared-memory addresses
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* Bs = base;                       // W2, swizzled K-major, 256 rows
  unsigned char* As = Bs + kBBytes;               // h1 tile, swizzled K-major, 128 rows
  float* b2s = (float*)(As + kABytes);
  float* w3s = b2s + kH;
  uint64_t* bar = (uint64_t*)(w3s + kH);
  uint32_t* tmem_slot = (uint32_t*)(bar + 1);
  float* partA = (float*)(tmem_slot + 14);        // [kTR][kPartStride] (16-byte aligned)
  float* partB = partA + kTR * kPartStride;       // [kTC][kPartStride]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ unsigned s_cnt[5];                   // kept pairs per warp of the tile, then the tile's base

  for (int e = tid; e < kH * (kH / 8); e += kTM) {          // W2 rows, 16 bytes at a time
    const int row = e >> 5, c16 = e & 31;
    *reinterpret_cast<uint4*>(Bs + swz(kH, row, c16)) = *reinterpret_cast<const uint4*>(g.W2b + row * kH + c16 * 8);
  }
  for (int j = tid; j < kH; j += kTM) {
    b2s[j] = g.b2[j];
    w3s[j] = g.w3[j];
  }
  if (tid == 0) mbar_init(bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kH)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // W2 visible to the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const float b3 = g.b3[0];
  const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
  unsigned phase = 0;
  bool mma_pending = false;

  for (int64_t t = blockIdx.x; t < g.n_tiles; t += gridDim.x) {
    const int ri = tile_rect(g.prefix, g.n_rects, t);
    const Rect rc = g.rects[ri];
    const int n_tc = (rc.w + kTC - 1) / kTC;
    const int64_t it = t - g.prefix[ri];
    const int row0 = (int)(it / n_tc) * kTR, col0 = (int)(it % n_tc) * kTC;
    const int row = row0 + (tid >> 4), col = col0 + (tid & 15);
    const bool valid = row < rc.rows && col < rc.w;
    const int64_t a = rc.ns0 + row, b = rc.r0 + col;
    const int64_t out = rc.out0 + (int64_t)row * rc.ld + col;
    const int mb = rc.n - rc.Ma;
    const bool model = rc.Ma <= kModelQp && mb <= kModelQp;     // uniform over the tile
    float y = 0.f;
    if (model) {
      // 0. the tile's partial rows (rows and columns beyond the rectangle: zeros, never used)
      for (int e = tid; e < (kTR + kTC) * (kH / 4); e += kTM) {
        const int q = e / (kH / 4), c4 = e - q * (kH / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < kTR) {
          if (row0 + q < rc.rows) v = __ldg(reinterpret_cast<const float4*>(g.Apart + (rc.ns0 + row0 + q) * kH) + c4);
          *reinterpret_cast<float4*>(partA + q * kPartStride + 4 * c4) = v;
        } else {
          const int qb = q - kTR;
          if (col0 + qb < rc.w) v = __ldg(reinterpret_cast<const float4*>(g.Bpart + (rc.r0 + col0 + qb) * kH) + c4);
          *reinterpret_cast<float4*>(partB + qb * kPartStride + 4 * c4) = v;
        }
      }
      __syncthreads();
      // 1. this pair's row of h1 = relu(A_a + B_b) in BF16
      const float4* ap = reinterpret_cast<const float4*>(partA + (tid >> 4) * kPartStride);
      const float4* bp = reinterpret_cast<const float4*>(partB + (tid & 15) * kPartStride);
#pragma unroll 4
      for (int c16 = 0; c16 < kH / 8; ++c16) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (valid) {
          const float4 a0 = ap[2 * c16], a1 = ap[2 * c16 + 1];
          const float4 b0 = bp[2 * c16], b1v = bp[2 * c16 + 1];
          v.x = pack2(fmaxf(a0.x + b0.x, 0.f), fmaxf(a0.y + b0.y, 0.f));
          v.y = pack2(fmaxf(a0.z + b0.z, 0.f), fmaxf(a0.w + b0.w, 0.f));
          v.z = pack2(fmaxf(a1.x + b1v.x, 0.f), fmaxf(a1.y + b1v.y, 0.f));
          v.w = pack2(fmaxf(a1.z + b1v.z, 0.f), fmaxf(a1.w + b1v.w, 0.f));
        }
        *reinterpret_cast<uint4*>(As + swz(kTM, tid, c16)) = v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // h1 visible to the tensor cores
      tc_fence_before();
      __syncthreads();
      // 2. layer 2: 16 MMAs of K = 16 (32 bytes of each 128-byte row per step)
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < kH / 16; ++s) {
          const uint32_t koff = (uint32_t)((s & 3) * 32);
          const uint64_t ad = sdesc(a_base + (uint32_t)(s >> 2) * (kTM * 128) + koff);
          const uint64_t bd = sdesc(b_base + (uint32_t)(s >> 2) * (kH * 128) + koff);
          tc_mma(tmem, ad, bd, kIdesc, s > 0 ? 1u : 0u);
        }
        tc_commit(bar);
      }
      const bool done = mbar_wait(bar, phase);
      if (__syncthreads_or(!done)) {                  // every thread leaves together
        if (tid == 0) atomicOr(g.status, kStTimeout);
        mma_pending = true;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
      // 3. layer 3 from this thread's accumulator row (TMEM lane = tid)
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
      float acc = 0.f;
#pragma unroll 1
      for (int c0 = 0; c0 < kH; c0 += 32) {
        float v[32];
        tc_ld32(lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc = fmaf(fmaxf(v[j] + b2s[c0 + j], 0.f), w3s[c0 + j], acc);
      }
      y = acc + b3;
      tc_fence_before();
    }
    // 4. decision, prediction, compaction
    if (valid && g.pred) g.pred[out - g.pred_base] = y;
    if (g.counts) {                                   // one atomic per tile (the tile has one size)
      const bool keep = valid && (!model || y - g.half_log_l * (float)rc.n + g.shift >= 0.f);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) s_cnt[warp] = (unsigned)__popc(m);
      __syncthreads();
      if (tid == 0) {
        const unsigned tot = s_cnt[0] + s_cnt[1] + s_cnt[2] + s_cnt[3];
        s_cnt[4] = tot ? atomicAdd(g.counts + (rc.n >> 1), tot) : 0u;
      }
      __syncthreads();
      if (keep) {
        unsigned before = s_cnt[4];
        for (int w = 0; w < warp; ++w) before += s_cnt[w];
        const int64_t slot = g.list_off[rc.n >> 1] + before + __popc(m & ((1u << lane) - 1u));
        g.lists[slot] = PairEntry{out, (int32_t)a, (int32_t)b};
      }
    }
    __syncthreads();                                   // the tile's h1 and accumulator are done with
  }
  if (mma_pending) mbar_wait(bar, phase);              // after a timeout: let the MMAs finish (bounded)
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kH) : "memory");
  }
}

}  // namespace

size_t score_tc_smem() { return kSmemBytes; }

// Scores of the pairs of the given rectangles (any sectors), see the file header.  Apart/Bpart:
// per-state partials over all states of the basis (global indices).
tgba_status score_rects_tc(Basis& b, const std::vector<Rect>& rects, const float* Apart, const float* Bpart,
                           const __nv_bfloat16* W2b, const float* b2, const float* w3, const float* b3, float shift,
                           float half_log_l, float* pred, int64_t pred_base, unsigned* counts,
                           const int64_t* list_off, PairEntry* lists, cudaStream_t st) {
  if (rects.empty()) return TGBA_OK;
  std::vector<int64_t> prefix(rects.size() + 1, 0);
  for (size_t i = 0; i < rects.size(); ++i)
    prefix[i + 1] = prefix[i] + (int64_t)((rects[i].rows + kTR - 1) / kTR) * ((rects[i].w + kTC - 1) / kTC);
  const int64_t n_tiles = prefix.back();
  if (n_tiles == 0) return TGBA_OK;
  void* buf = nullptr;
  const size_t rb = rects.size() * sizeof(Rect), pb = prefix.size() * sizeof(int64_t);
  TGBA_CUDA(cudaMallocAsync(&buf, rb + pb, st));
  TGBA_CUDA(cudaMemcpyAsync(buf, rects.data(), rb, cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemcpyAsync((char*)buf + rb, prefix.data(), pb, cudaMemcpyHostToDevice, st));
  ScoreArgs g;
  g.rects = (const Rect*)buf;
  g.prefix = (const int64_t*)((char*)buf + rb);
  g.n_rects = (int)rects.size();
  g.n_tiles = n_tiles;
  g.Apart = Apart; g.Bpart = Bpart; g.W2b = W2b; g.b2 = b2; g.w3 = w3; g.b3 = b3;
  g.shift = shift; g.half_log_l = half_log_l;
  g.pred = pred; g.pred_base = pred_base;
  g.counts = counts; g.list_off = list_off; g.lists = lists;
  g.status = b.d_status;
  TGBA_CUDA(cudaFuncSetAttribute(score_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  int sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  const int grid = (int)std::min<int64_t>(n_tiles, sms);
  score_tc<<<grid, kTM, kSmemBytes, st>>>(g);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  TGBA_CUDA(cudaFreeAsync(buf, st));
  return TGBA_OK;
}

}  // namespace tgba
