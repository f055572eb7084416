// Batched Pfaffians of the Pfaffian stage (row a4 of the hot path; Appendix A, Eq. S1-S2, S4).
//
// Element (a, b) of a sector: sel = (table rows of a's NS excitation operators, ascending) ++
// (table rows of b's R excitation operators, ascending), n = M_a + M_b, and
//     P_ab = Pf(R[sel, sel]),   X_ab = C0 (-i)^{n/2} P_ab
// with R the real contraction table.  Pf is computed by Parlett-Reid reduction with partial
// pivoting in FP64, one thread per element.  The n x n strict upper triangle lives in shared
// memory laid out [entry][thread], so the 32 lanes of a warp touch 32 consecutive doubles.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the kernel is bound by the FP64 pipe alone: the
// per-step pivot search compares magnitudes as integers (the bit pattern of |x|), index
// arithmetic and shared-memory traffic are integer/LSU work, and only the elimination itself
// (one FMA pair per updated entry, one multiply per Gauss-vector entry, one reciprocal and one
// multiply per step) issues FP64 instructions.
//
// Work: tiles of up to THREADS elements with uniform n (see build_tiles), grouped in size
// classes; one persistent launch per class walks its tiles with a grid-stride loop.  Sizes
// n <= 14 run the register-resident kernel of pfaffian_reg.cuh, one class per exact n; larger
// sizes run the shared-memory kernel below.
#include <algorithm>

#include "pfaffian_reg.cuh"
#include "tgba_internal.h"

namespace tgba {

namespace {

template <int NMAX>
struct Packed {
  // strict upper triangle of an NMAX x NMAX matrix, row-major
  static __device__ __forceinline__ int idx(int i, int j) { return i * (2 * NMAX - i - 1) / 2 + (j - i - 1); }
  static constexpr int kEntries = NMAX * (NMAX - 1) / 2;
};

__device__ __forceinline__ unsigned long long mag(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Pf of the n x n skew matrix whose strict upper triangle is in W (packed, stride T).
template <int NMAX, int T>
__device__ double pfaffian_smem(double* W, int n) {
  using P = Packed<NMAX>;
  double pf = 1.0;
  for (int k = 0; k + 1 < n; k += 2) {
    const int r = k + 1;
    // pivot: largest |W(k, x)|, x > k
    int p = r;
    unsigned long long best = mag(W[P::idx(k, r) * T]);
    for (int x = r + 1; x < n; ++x) {
      unsigned long long v = mag(W[P::idx(k, x) * T]);
      if (v > best) { best = v; p = x; }
    }
    if (p != r) {
      // symmetric exchange of rows/columns r and p, restricted to rows >= k
      double t = W[P::idx(k, r) * T]; W[P::idx(k, r) * T] = W[P::idx(k, p) * T]; W[P::idx(k, p) * T] = t;
      for (int x = r + 1; x < p; ++x) {
        double a = W[P::idx(r, x) * T], c = W[P::idx(x, p) * T];
        W[P::idx(r, x) * T] = -c;
        W[P::idx(x, p) * T] = -a;
      }
      W[P::idx(r, p) * T] = -W[P::idx(r, p) * T];
      for (int x = p + 1; x < n; ++x) {
        double a = W[P::idx(r, x) * T];
        W[P::idx(r, x) * T] = W[P::idx(p, x) * T];
        W[P::idx(p, x) * T] = a;
      }
      pf = -pf;
    }
    const double a = W[P::idx(k, r) * T];
    if (a == 0.0) return 0.0;          // the whole column is zero: Pf = 0 exactly
    pf *= a;
    if (k + 2 >= n) break;
    const double ia = 1.0 / a;
    for (int j = k + 2; j < n; ++j) W[P::idx(k, j) * T] *= ia;     // Gauss vector tau_j
    // trailing update: W_ij += W(r, i) tau_j - tau_i W(r, j),  k+2 <= i < j < n
    for (int i = k + 2; i < n - 1; ++i) {
      const double a1i = W[P::idx(r, i) * T];
      const double ti = W[P::idx(k, i) * T];
      const int base = P::idx(i, i + 1);
      const int rk = P::idx(k, i + 1), rr = P::idx(r, i + 1);
#pragma unroll 4
      for (int j = i + 1; j < n; ++j) {
        const int o = j - i - 1;
        double w = W[(base + o) * T];
        w = fma(-ti, W[(rr + o) * T], w);
        w = fma(a1i, W[(rk + o) * T], w);
        W[(base + o) * T] = w;
      }
    }
  }
  return pf;
}

template <int NMAX, int T>
__global__ void __launch_bounds__(T) pf_tiles(const Tile* __restrict__ tiles, int t_begin, int t_end,
                                              const double* __restrict__ R, int two_l,
                                              const uint8_t* __restrict__ sel_ns, const uint8_t* __restrict__ sel_r,
                                              int max_qp, const uint8_t* __restrict__ mask, double* __restrict__ P,
                                              unsigned* status) {
  extern __shared__ double smem[];
  double* W = smem + threadIdx.x;
  for (int t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
    const Tile tl = tiles[t];
    const int e = threadIdx.x;
    if (e >= tl.count) continue;
    const int lin = tl.lin0 + e;
    const int row = lin / tl.w, col = lin - (lin / tl.w) * tl.w;
    const int64_t out = tl.out0 + (int64_t)row * tl.ld + col;
    if (mask != nullptr && mask[out] == 0) { P[out] = 0.0; continue; }
    const int n = tl.n, ma = tl.Ma;
    const uint8_t* sa = sel_ns + (size_t)(tl.ns0 + row) * max_qp;
    const uint8_t* sb = sel_r + (size_t)(tl.r0 + col) * max_qp;
    // gather R[sel_i][sel_j], i < j, from the (L2-resident) table
    for (int i = 0; i < n - 1; ++i) {
      const int si = i < ma ? sa[i] : sb[i - ma];
      const double* Ri = R + (size_t)si * two_l;
      for (int j = i + 1; j < n; ++j) {
        const int sj = j < ma ? sa[j] : sb[j - ma];
        W[Packed<NMAX>::idx(i, j) * T] = __ldg(Ri + sj);
      }
    }
    const double pf = pfaffian_smem<NMAX, T>(W, n);
    if (!isfinite(pf)) atomicOr(status, kStNan);
    P[out] = pf;
  }
}

// Register-resident variant for one exact size N <= 14 (see pfaffian_reg.cuh).
template <int N, int T>
__global__ void __launch_bounds__(T) pf_tiles_reg(const Tile* __restrict__ tiles, int t_begin, int t_end,
                                                  const double* __restrict__ R, int two_l,
                                                  const uint8_t* __restrict__ sel_ns, const uint8_t* __restrict__ sel_r,
                                                  int max_qp, const uint8_t* __restrict__ mask, double* __restrict__ P,
                                                  unsigned* status) {
  for (int t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
    const Tile tl = tiles[t];
    const int e = threadIdx.x;
    if (e >= tl.count) continue;
    const int lin = tl.lin0 + e;
    const int row = lin / tl.w, col = lin - (lin / tl.w) * tl.w;
    const int64_t out = tl.out0 + (int64_t)row * tl.ld + col;
    if (mask != nullptr && mask[out] == 0) { P[out] = 0.0; continue; }
    if constexpr (N == 0) {
      P[out] = 1.0;
    } else {
      const int ma = tl.Ma;
      const uint8_t* sa = sel_ns + (size_t)(tl.ns0 + row) * max_qp;
      const uint8_t* sb = sel_r + (size_t)(tl.r0 + col) * max_qp;
      int sel[N];
#pragma unroll
      for (int i = 0; i < N; ++i) sel[i] = i < ma ? sa[i] : sb[i - ma];
      double W[N][N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double* Ri = R + (size_t)sel[i] * two_l;
#pragma unroll
        for (int j = i + 1; j < N; ++j) W[i][j] = __ldg(Ri + sel[j]);
      }
      const double pf = pfaffian_regs<N>(W);
      if (!is_finite_bits(pf)) atomicOr(status, kStNan);
      P[out] = pf;
    }
  }
}

// One thread per explicit (a, b) pair; sizes vary per thread.
template <int NMAX, int T>
__global__ void __launch_bounds__(T) pf_pairs(const int32_t* __restrict__ pairs, int64_t n_pairs, int64_t ns_off,
                                              int64_t r_off, int64_t n_ns, int64_t n_r,
                                              const double* __restrict__ R, int two_l,
                                              const uint8_t* __restrict__ sel_ns, const uint8_t* __restrict__ sel_r,
                                              const uint8_t* __restrict__ m_ns, const uint8_t* __restrict__ m_r,
                                              int max_qp, const double* __restrict__ c0, double* __restrict__ out,
                                              unsigned* status) {
  extern __shared__ double smem[];
  double* W = smem + threadIdx.x;
  for (int64_t q = (int64_t)blockIdx.x * T + threadIdx.x; q < n_pairs; q += (int64_t)gridDim.x * T) {
    const int32_t pa = pairs[2 * q], pb = pairs[2 * q + 1];
    if (pa < 0 || pa >= n_ns || pb < 0 || pb >= n_r) {      // reject, never read out of range
      atomicOr(status, kStBadIndex);
      out[2 * q] = out[2 * q + 1] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const int64_t a = ns_off + pa, b = r_off + pb;
    const int ma = m_ns[a], n = ma + m_r[b];
    const uint8_t* sa = sel_ns + (size_t)a * max_qp;
    const uint8_t* sb = sel_r + (size_t)b * max_qp;
    for (int i = 0; i < n - 1; ++i) {
      const int si = i < ma ? sa[i] : sb[i - ma];
      for (int j = i + 1; j < n; ++j) {
        const int sj = j < ma ? sa[j] : sb[j - ma];
        W[Packed<NMAX>::idx(i, j) * T] = __ldg(R + (size_t)si * two_l + sj);
      }
    }
    const double pf = pfaffian_smem<NMAX, T>(W, n);
    if (!isfinite(pf)) atomicOr(status, kStNan);
    // X = C0 (-i)^{n/2} pf
    double re = c0[0] * pf, im = c0[1] * pf;
    switch ((n / 2) & 3) {
      case 0: out[2 * q] = re; out[2 * q + 1] = im; break;
      case 1: out[2 * q] = im; out[2 * q + 1] = -re; break;
      case 2: out[2 * q] = -re; out[2 * q + 1] = -im; break;
      default: out[2 * q] = -im; out[2 * q + 1] = re; break;
    }
  }
}

template <int NMAX, int T>
tgba_status launch_class(Basis& b, int t0, int t1, const uint8_t* mask, cudaStream_t st) {
  if (t1 <= t0) return TGBA_OK;
  const size_t smem = (size_t)Packed<NMAX>::kEntries * T * sizeof(double);
  auto kern = pf_tiles<NMAX, T>;
  TGBA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  TGBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem));
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  if (per_sm < 1) return fail(TGBA_ELIMIT, "Pfaffian kernel does not fit on an SM");
  const int grid = std::min(t1 - t0, per_sm * sms);
  kern<<<grid, T, smem, st>>>(b.d_tiles, t0, t1, b.d_table, 2 * b.L, b.d_sel_ns, b.d_sel_r, b.max_qp, mask, b.d_P,
                              b.d_status);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

template <int N>
tgba_status launch_reg(Basis& b, int t0, int t1, const uint8_t* mask, cudaStream_t st) {
  if (t1 <= t0) return TGBA_OK;
  constexpr int T = 128;
  auto kern = pf_tiles_reg<N, T>;
  TGBA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
  int per_sm = 0, sms = 0;
  TGBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, 0));
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  if (per_sm < 1) return fail(TGBA_ELIMIT, "register Pfaffian kernel does not fit on an SM");
  const int grid = std::min(t1 - t0, per_sm * sms);
  kern<<<grid, T, 0, st>>>(b.d_tiles, t0, t1, b.d_table, 2 * b.L, b.d_sel_ns, b.d_sel_r, b.max_qp, mask, b.d_P,
                           b.d_status);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

template <int NMAX, int T>
tgba_status launch_pairs(Basis& b, int s, const int32_t* pairs, int64_t n, double* out, cudaStream_t st) {
  const size_t smem = (size_t)Packed<NMAX>::kEntries * T * sizeof(double);
  auto kern = pf_pairs<NMAX, T>;
  TGBA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  const int64_t blocks = std::min<int64_t>((n + T - 1) / T, (int64_t)sms * 8);
  const Sector& sec = b.sectors[s];
  kern<<<(int)blocks, T, smem, st>>>(pairs, n, sec.ns_off, sec.r_off, sec.n_ns, sec.n_r, b.d_table, 2 * b.L, b.d_sel_ns, b.d_sel_r,
                                     b.d_M_ns, b.d_M_r, b.max_qp, b.d_c0, out, b.d_status);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

}  // namespace

tgba_status run_pfaffians(Basis& b, const uint8_t* mask, cudaStream_t st) {
  const std::vector<int>& cb = b.tile_class_begin;
  tgba_status r;
  // one launch per size class, largest Pfaffians first (class layout: see tile_class)
  if ((r = launch_class<32, 32>(b, cb[11], cb[12], mask, st)) != TGBA_OK) return r;
  if ((r = launch_class<24, 64>(b, cb[10], cb[11], mask, st)) != TGBA_OK) return r;
  if ((r = launch_class<20, 128>(b, cb[9], cb[10], mask, st)) != TGBA_OK) return r;
  if ((r = launch_class<16, 128>(b, cb[8], cb[9], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<14>(b, cb[7], cb[8], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<12>(b, cb[6], cb[7], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<10>(b, cb[5], cb[6], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<8>(b, cb[4], cb[5], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<6>(b, cb[3], cb[4], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<4>(b, cb[2], cb[3], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<2>(b, cb[1], cb[2], mask, st)) != TGBA_OK) return r;
  if ((r = launch_reg<0>(b, cb[0], cb[1], mask, st)) != TGBA_OK) return r;
  return TGBA_OK;
}

tgba_status run_pfaffian_pairs(Basis& b, int s, const int32_t* pairs, int64_t n, double* out, cudaStream_t st) {
  if (n == 0) return TGBA_OK;
  if (b.max_n <= 12) return launch_pairs<12, 128>(b, s, pairs, n, out, st);
  if (b.max_n <= 20) return launch_pairs<20, 64>(b, s, pairs, n, out, st);
  return launch_pairs<32, 32>(b, s, pairs, n, out, st);
}

}  // namespace tgba
