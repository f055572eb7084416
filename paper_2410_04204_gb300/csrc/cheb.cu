// Batched Chebyshev propagation of the quench variants (row a9: Eq. 10 and the norm statement
// of the Quench section).
//
// Every variant v keeps a prefix of one ranking of the sector's NS states and a prefix of one
// ranking of its R states (nested truncations) and has its own longitudinal field h_x,v.  In
// the real gauge of H_eff,
//   H~_v = D + g_v A,  D = diag(E^(0)),  A = [[0, Q^T], [Q, 0]],  g_v = -L h_x,v |C0|,
// with Q the real X block of the kept states (R rows, NS columns).  B(t) = e^{-iH~t} c~0 is
// expanded in Chebyshev polynomials of H' = (H~ - E_c)/R by the Jacobi-Anger identity,
//   B(t) = e^{-i E_c t} sum_k (2 - d_k0) (-i)^k J_k(R t) v_k,   v_k = T_k(H') c~0,
// and because sigma^x_1 is the off-diagonal part of H_eff, X~ = (D - H~)/(L h_x), so the
// magnetisation needs only moments weighted by the diagonal:
//   B^H X~ B = ( B^H (D - E_c) B - c~0^H (H~ - E_c) c~0 ) / (L h_x),
//   B^H (D - E_c) B = sum_kl a_k a_l Re(i^{k-l} v_k^H (D - E_c) v_l),  a_k = (2 - d_k0) J_k(R t),
//   c~0^H (H~ - E_c) c~0 = R Re(v_0^H v_1)      (the energy is conserved),
// and <sigma^x>(t) = B^H X~ B / ||c0||^2.  The moments take 6 K^2 chi flops per variant instead
// of the 2 chi^2 K of v_k^H X~ v_l.  Absolute error of <sigma^x>: about K eps R / (L |h_x|).
//
// The interval [E_c - R, E_c + R] comes from Lanczos: 64 steps on the union of the kept states
// (the largest variant) for each distinct h_x give the extreme Ritz values, widened by 2%; by
// Cauchy interlacing every nested variant's spectrum lies inside.  The bound is checked after
// the propagation: with the spectrum inside, ||v_K|| <= ||v_0||, while any part outside grows
// like cosh(K acosh|x|); if the check fails the propagation is redone with Gershgorin bounds.
//
// Layout: all variants' vectors side by side on the union of the kept states (NS rows, then R
// rows), two real columns (Re, Im of c~0's propagation) per variant, variants ordered by
// decreasing kept set; entries outside a variant's set stay 0.  Every FP64 product (the
// off-diagonal blocks in each step, the Lanczos steps and the moments) runs on the tensor cores
// through the sliced products of dgemm_tc.cu: Q is sliced once in both orientations, each
// step slices the current vectors, and the output tiles of each step skip the (row block,
// column block) pairs that no variant's kept set reaches.  The K steps are captured into one
// CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "tgba_internal.h"

namespace tgba {
namespace {

constexpr int kLanczosSteps = 64;
constexpr int kRedThreads = 1024;

__device__ __forceinline__ double block_reduce(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += sh[w];   // fixed order: every thread gets the same value
  return s;
}

// dst (cols x rows, row-major) = transpose of src (rows x cols, row-major), 32 x 32 tiles
__global__ void transpose_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, double* __restrict__ dst) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = src[r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[c * rows + r] = t[threadIdx.x][i];
  }
}

// Lanczos start vectors: a fixed pseudo-random vector per column (SplitMix64 of the row), unit norm
__global__ void lz_start(int64_t n, double* __restrict__ q) {
  __shared__ double sh[32];
  double* col = q + (int64_t)blockIdx.x * n;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    unsigned long long z = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull + (unsigned long long)blockIdx.x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double v = (double)(z >> 11) * 0x1p-53 - 0.5;
    col[i] = v;
    s = fma(v, v, s);
  }
  s = block_reduce(s, sh);
  const double inv = 1.0 / sqrt(s);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) col[i] *= inv;
}

// One Lanczos step per column (block): w = g Y + E q; alpha = q.w; w -= alpha q + beta q_prev;
// beta' = ||w||; q_next = w / beta' (zero after a breakdown).  Y holds A q.
__global__ void lz_step(int64_t n, const double* __restrict__ E, const double* __restrict__ g, const double* __restrict__ Y,
                        const double* __restrict__ qp, const double* __restrict__ qc, double* __restrict__ qn,
                        double* __restrict__ alpha, double* __restrict__ beta, int j, int m) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const double gc = g[c];
  const double* y = Y + (int64_t)c * n;
  const double* p = qp + (int64_t)c * n;
  const double* q = qc + (int64_t)c * n;
  double* w = qn + (int64_t)c * n;
  const double b_j = j > 0 ? beta[(int64_t)c * m + j] : 0.0;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = fma(gc, y[i], E[i] * q[i]);
    w[i] = v;
    s = fma(q[i], v, s);
  }
  const double a = block_reduce(s, sh);
  s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = w[i] - a * q[i] - b_j * p[i];
    w[i] = v;
    s = fma(v, v, s);
  }
  const double bn = sqrt(block_reduce(s, sh));
  const double inv = bn > 1e-300 ? 1.0 / bn : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) w[i] *= inv;
  if (threadIdx.x == 0) {
    alpha[(int64_t)c * m + j] = a;
    if (j + 1 < m) beta[(int64_t)c * m + j + 1] = bn;
  }
}

// Row sums of |Q| (Q: col-major kr x kn, ld kr): rs[a] for NS column a, rs[kn + b] for R row b.
__global__ void abs_sums_ns(int64_t kn, int64_t kr, const double* __restrict__ Q, double* __restrict__ rs) {
  const int lane = threadIdx.x & 31;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < kn; a += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int64_t b = lane; b < kr; b += 32) s += fabs(Q[a * kr + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rs[a] = s;
  }
}
__global__ void abs_sums_r(int64_t kn, int64_t kr, const double* __restrict__ Q, double* __restrict__ rs) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < kr; b += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t a = 0; a < kn; ++a) s += fabs(Q[a * kr + b]);
    rs[kn + b] = s;
  }
}

// Per column of the union layout: coupling g, centre E_c, 1/R, and the kept set (kn NS rows
// from 0, kr R rows from kn_max).  Padding columns have kn = kr = 0 and stay 0.
struct ColPrm {
  double g, ec, invr;
  int64_t kn, kr;
};

__device__ __forceinline__ bool kept(int64_t row, int64_t kn_max, const ColPrm& p) {
  return row < kn_max ? row < p.kn : row - kn_max < p.kr;
}

// v_0: column 2j = Re c~0, 2j + 1 = Im c~0 on the kept rows of its variant
__global__ void cheb_init(int64_t n, int64_t kn_max, int cols, const ColPrm* __restrict__ prm,
                          const double* __restrict__ c, double* __restrict__ V) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * cols; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q % n;
    const int col = (int)(q / n);
    V[q] = kept(row, kn_max, prm[col]) ? c[2 * row + (col & 1)] : 0.0;
  }
}

// v_{k+1} = alpha (g Y + (E - E_c) v_k) / R - beta v_{k-1}, 0 outside each column's kept rows
__global__ void cheb_step(int64_t n, int64_t kn_max, int cols, const double* __restrict__ E,
                          const ColPrm* __restrict__ prm, double alpha, double beta, const double* __restrict__ Y,
                          const double* __restrict__ x, const double* __restrict__ prev, double* __restrict__ next) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * cols; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q % n;
    const ColPrm p = prm[q / n];
    double v = 0.0;
    if (kept(row, kn_max, p)) {
      const double h = fma(p.g, Y[q], (E[row] - p.ec) * x[q]);
      v = alpha * p.invr * h - (prev ? beta * prev[q] : 0.0);
    }
    next[q] = v;
  }
}

// per column: ||v_0||^2 and ||v_K||^2 (one block per column)
__global__ void cheb_norms(int64_t n, const double* __restrict__ V0, const double* __restrict__ VK,
                           double* __restrict__ out) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  double s0 = 0.0, sk = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = V0[(int64_t)c * n + i], b = VK[(int64_t)c * n + i];
    s0 = fma(a, a, s0);
    sk = fma(b, b, sk);
  }
  s0 = block_reduce(s0, sh);
  sk = block_reduce(sk, sh);
  if (threadIdx.x == 0) { out[2 * c] = s0; out[2 * c + 1] = sk; }
}

// energies of a kept set in its own order: kn NS rows, then kr R rows
__global__ void kept_energy(int64_t kn, int64_t kr, int64_t kn_max, const double* __restrict__ E, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kn + kr; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < kn ? E[i] : E[kn_max + (i - kn)];
}

// Re(v_0^H v_1) of one variant (columns c, c + 1 of v_0 and of v_1)
__global__ void cheb_dot01(int64_t n, const double* __restrict__ v0, const double* __restrict__ v1, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(v0[i], v1[i], fma(v0[n + i], v1[n + i], s));
  s = block_reduce(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// Gamma_kl = Re(i^{k-l} mu_kl), mu = (G_rr + G_ii) + i (G_ri - G_ri^T), G column-major K1 x K1;
// G_rr and G_ii are symmetric and only their lower triangle (row >= column) is computed
__global__ void cheb_gamma(int K1, const double* __restrict__ Grr, const double* __restrict__ Gii,
                           const double* __restrict__ Gri, double* __restrict__ Gam) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)K1 * K1; q += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(q / K1), k = (int)(q % K1);
    const int64_t kl = (int64_t)l * K1 + k, lk = (int64_t)k * K1 + l;
    const int64_t low = k >= l ? kl : lk;
    const double re = Grr[low] + Gii[low], im = Gri[kl] - Gri[lk];
    double g;
    switch (((k - l) % 4 + 4) % 4) {
      case 0: g = re; break;
      case 1: g = -im; break;
      case 2: g = -re; break;
      default: g = im; break;
    }
    Gam[kl] = g;
  }
}

// a_k(t) = (2 - d_k0) J_k(R t), k = 0..K, by Miller's backward recurrence for J_k
// (J_{k-1} = (2k/x) J_k - J_{k+1} from a start far above k and x, normalised by
// J_0 + 2 sum J_2j = 1), one thread per time.  out is [k][t] (row k at out + k n_t), so a
// warp's stores of one k are consecutive; 2k/x is 2k times 1/x, taken once (no FP64 division
// in the recurrence).  When the unnormalised values pass 1e250 the recurrence is rescaled by
// 1e-250 without touching the values already stored: an entry stored before one rescaling
// gets the factor 1e-250 at the end, one stored before two or more is below 1e-236 of the
// result and becomes 0, so only the positions of the last two rescalings are kept.
__global__ void cheb_bessel(int n_t, int t0, double dt, double R, int K, int m_start, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_t) return;
  const double x = R * dt * (double)(t0 + c);
  double* a = out + c;                         // a_k at a[k n_t]
  const int64_t S = n_t;
  if (x == 0.0) {
    a[0] = 1.0;
    for (int k = 1; k <= K; ++k) a[k * S] = 0.0;
    return;
  }
  const double ix2 = 2.0 / x;
  double jp1 = 0.0, j = 1e-300, norm = 0.0;
  int k_last = 1 << 30, k_prev = 1 << 30;     // the last two rescalings (entry q was stored before
                                               // the one at k iff q + 1 >= k)
  for (int k = m_start; k >= 1; --k) {
    const double jm1 = fma((double)k * ix2, j, -jp1);
    jp1 = j;
    j = jm1;                                   // j = J_{k-1} (unnormalised)
    if (k - 1 <= K) a[(k - 1) * S] = j;
    if ((k - 1) % 2 == 0 && k - 1 > 0) norm += 2.0 * j;
    if (fabs(j) > 1e250) {
      const double sc = 1e-250;
      j *= sc; jp1 *= sc; norm *= sc;
      k_prev = k_last;
      k_last = k;
    }
  }
  norm += j;                                   // + J_0
  const double inv = 1.0 / norm;
  for (int q = 0; q <= K; ++q) {
    const double f = (q + 1 >= k_prev) ? 0.0 : (q + 1 >= k_last ? 1e-250 : 1.0);
    a[q * S] *= (q == 0 ? inv : 2.0 * inv) * f;
  }
}

// mx[t] = (a(t)^T Gamma a(t) - e_shift) * scale, one warp per time (A = a [k][t], GA = Gamma a
// precomputed, [t][k])
__global__ void cheb_mx(int K1, int cnt, const double* __restrict__ A, const double* __restrict__ GA, double e_shift,
                        double scale, double* __restrict__ mx) {
  const int lane = threadIdx.x & 31;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= cnt) return;
  double acc = 0.0;
  for (int k = lane; k < K1; k += 32) acc = fma(A[(int64_t)k * cnt + col], GA[(int64_t)col * K1 + k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) mx[col] = (acc - e_shift) * scale;
}

int blocks_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

// extreme eigenvalues of the symmetric tridiagonal matrix (a [m], b [m] with b[0] unused) by
// bisection on Sturm counts
void tridiag_extremes(const double* a, const double* b, int m, double* lo, double* hi) {
  double g0 = 1e300, g1 = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < m ? std::fabs(b[i + 1]) : 0.0);
    g0 = std::min(g0, a[i] - r);
    g1 = std::max(g1, a[i] + r);
  }
  auto count = [&](double x) {              // eigenvalues below x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = (a[i] - x) - (i > 0 ? b[i] * b[i] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++c;
    }
    return c;
  };
  auto kth = [&](int k) {
    double l = g0, h = g1;
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(1.0, std::fabs(l) + std::fabs(h)); ++it) {
      const double mid = 0.5 * (l + h);
      if (count(mid) <= k) l = mid;
      else h = mid;
    }
    return 0.5 * (l + h);
  };
  *lo = kth(0);
  *hi = kth(m - 1);
}

struct DevBuf {
  void* p = nullptr;
  cudaStream_t s;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  ~DevBuf() { if (p) cudaFreeAsync(p, s); }
};

int64_t r16(int64_t x) { return (x + 15) / 16 * 16; }

// Output tiles of one off-diagonal product: rows (row blocks of 128) x the vector columns (blocks
// of 128).  Column c needs output rows below out_c[c] and K values below k_c[c]; a tile keeps the
// columns up to the last one that needs any of its rows, the K range they need, and per group of
// 16 columns the K range of its columns that need the tile's rows (one K block for a group with
// none).
std::vector<EmuTile> product_tiles(int64_t rows, int64_t cols, const std::vector<int64_t>& out_c,
                                   const std::vector<int64_t>& k_c) {
  const int TR = emu_tile_rows_a(), TC = emu_tile_rows_b(), KB = emu_k_block();
  std::vector<EmuTile> t;
  for (int64_t rb = 0; rb * TR < rows; ++rb)
    for (int64_t cb = 0; cb * TC < cols; ++cb) {
      int64_t last = -1, kmax = 0, kg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int64_t c = cb * TC; c < std::min(cols, (cb + 1) * TC); ++c)
        if (out_c[c] > rb * TR && k_c[c] > 0) {
          last = c - cb * TC;
          kmax = std::max(kmax, k_c[c]);
          kg[last / 16] = std::max(kg[last / 16], k_c[c]);
        }
      if (last < 0) continue;
      EmuTile e{(int32_t)rb, (int32_t)cb, (int32_t)std::min<int64_t>(TC, r16(last + 1)),
                (int32_t)((kmax + KB - 1) / KB)};
      for (int q = 0; q < 8; ++q) e.gkb[q] = (int16_t)std::max<int64_t>(1, (kg[q] + KB - 1) / KB);
      t.push_back(e);
    }
  return t;
}

}  // namespace

tgba_status quench_cheb_batch(Basis& b, const double* Q, int64_t kn_max, int64_t kr_max, const double* E,
                              const double* c, const std::vector<ChebVariant>& vars, double t_max, int n_t,
                              double* mx, cudaStream_t st) {
  if (vars.empty()) return TGBA_OK;
  for (const ChebVariant& v : vars)
    if (!(std::fabs(v.hx) * b.L >= 1e-3))
      return fail(TGBA_EINVAL, "the Chebyshev quench path needs |h_x| L >= 1e-3 (it reads <sigma^x> off the energy); "
                               "use method 1 for h_x = 0");
  const int64_t n_un = kn_max + kr_max;
  const double cabs = std::hypot(b.c0_host[0], b.c0_host[1]);
  const int TR = emu_tile_rows_a(), TC = emu_tile_rows_b();
  // stage times (host clock around synchronised sections)
  using clk = std::chrono::steady_clock;
  TGBA_CUDA(cudaStreamSynchronize(st));
  const auto t_start = clk::now();
  auto ms_since = [](clk::time_point t0) { return std::chrono::duration<double, std::milli>(clk::now() - t0).count(); };
  b.quench_prep_ms = b.quench_gram_ms = b.quench_eval_ms = 0.0;
  tgba_status r = emu_prepare(b);
  if (r != TGBA_OK) return r;
  // ---- Q sliced in both orientations: A_ns (NS rows, K = R) and A_r (R rows, K = NS)
  DevBuf qbuf(st);
  const size_t ens = emu_operand_elems((int)kn_max, (int)std::max<int64_t>(1, kr_max), TR);
  const size_t er = emu_operand_elems((int)kr_max, (int)std::max<int64_t>(1, kn_max), TR);
  const bool coupled = kn_max > 0 && kr_max > 0;
  TGBA_CUDA(cudaMallocAsync(&qbuf.p, (ens + er) * 2 + (size_t)(n_un + 16) * 4 + 256, st));
  __nv_bfloat16* A_ns = (__nv_bfloat16*)qbuf.p;
  __nv_bfloat16* A_r = A_ns + ens;
  int* e_ns = (int*)(A_r + er);
  int* e_r = e_ns + kn_max;
  if (coupled) {
    if ((r = emu_slice(b, Q, kr_max, 1, (int)kr_max, 0, nullptr, 0.0, (int)kn_max, (int)kr_max, TR, A_ns, e_ns, st)) !=
        TGBA_OK)
      return r;
    double* Qt = nullptr;                               // R rows, NS contiguous
    TGBA_CUDA(cudaMallocAsync(&Qt, (size_t)kn_max * kr_max * sizeof(double), st));
    transpose_kernel<<<dim3((unsigned)((kr_max + 31) / 32), (unsigned)((kn_max + 31) / 32)), dim3(32, 8), 0, st>>>(
        kn_max, kr_max, Q, Qt);
    ++b.launches;
    r = emu_slice(b, Qt, kn_max, 1, (int)kn_max, 0, nullptr, 0.0, (int)kr_max, (int)kn_max, TR, A_r, e_r, st);
    cudaFreeAsync(Qt, st);
    if (r != TGBA_OK) return r;
  }
  // B-operand slices of the current vectors (the columns padded to whole tiles)
  auto vec_slices = [&](int cols) {
    return std::max(emu_operand_elems(cols, (int)std::max<int64_t>(1, kr_max), TC),
                    emu_operand_elems(cols, (int)std::max<int64_t>(1, kn_max), TC));
  };
  // off-diagonal product Y = A x on the union layout (x, Y: n_un x cols, ld n_un)
  auto offdiag = [&](const double* x, double* Y, int cols, __nv_bfloat16* Bs, int* eb, EmuTile* t_ns, int n_ns,
                     int64_t c_ns, EmuTile* t_r, int n_r, int64_t c_r, int ns) -> tgba_status {
    tgba_status q = emu_slice(b, x + kn_max, n_un, 1, (int)kr_max, 0, nullptr, 0.0, cols, (int)kr_max, TC, Bs, eb, st);
    if (q == TGBA_OK) q = emu_gemm(b, A_ns, e_ns, (int)kn_max, (int)kr_max, Bs, eb, cols, (int)kr_max, t_ns, n_ns, c_ns, Y, n_un, st, ns);
    if (q == TGBA_OK) q = emu_slice(b, x, n_un, 1, (int)kn_max, 0, nullptr, 0.0, cols, (int)kn_max, TC, Bs, eb, st);
    if (q == TGBA_OK)
      q = emu_gemm(b, A_r, e_r, (int)kr_max, (int)kn_max, Bs, eb, cols, (int)kn_max, t_r, n_r, c_r, Y + kn_max, n_un, st, ns);
    return q;
  };
  // ---- Lanczos bounds on the union for each distinct field.  The products take only the two
  // leading digit slices of each operand (X's relative error about 2^-16 of its row scale, a
  // third of the slice traffic): the bounds are widened by 2% and checked after the
  // propagation, so they need the spectrum's edges to a few digits, not to FP64
  std::vector<double> fields;
  for (const ChebVariant& v : vars)
    if (std::find(fields.begin(), fields.end(), v.hx) == fields.end()) fields.push_back(v.hx);
  const int nh = (int)fields.size();
  const int nhp = (int)std::max<int64_t>(TC, (nh + TC - 1) / TC * TC);
  std::vector<double> lo(nh), hi(nh);
  {
    const int m = (int)std::min<int64_t>(kLanczosSteps, n_un);
    std::vector<int64_t> out_ns(nhp, 0), out_r(nhp, 0), k_ns(nhp, 0), k_r(nhp, 0);
    for (int i = 0; i < nh; ++i) { out_ns[i] = kn_max; k_ns[i] = kr_max; out_r[i] = kr_max; k_r[i] = kn_max; }
    std::vector<EmuTile> tn = product_tiles(kn_max, nhp, out_ns, k_ns), tr = product_tiles(kr_max, nhp, out_r, k_r);
    const int64_t cn = emu_number_tiles(tn), cr_ = emu_number_tiles(tr);
    if (cn < 0 || cr_ < 0) return fail(TGBA_EINVAL, "quench product tiles");
    DevBuf buf(st);
    const size_t vs = vec_slices(nhp);
    const size_t doubles = (size_t)4 * n_un * nhp + 2 * (size_t)m * nhp + nhp;
    const size_t tb = (tn.size() + tr.size()) * sizeof(EmuTile);
    TGBA_CUDA(cudaMallocAsync(&buf.p, doubles * 8 + vs * 2 + (size_t)nhp * 4 + tb + 512, st));
    double* q0 = (double*)buf.p;
    double* q1 = q0 + n_un * nhp;
    double* q2 = q1 + n_un * nhp;
    double* Y = q2 + n_un * nhp;
    double* al = Y + n_un * nhp;
    double* be = al + (size_t)m * nhp;
    double* g = be + (size_t)m * nhp;
    EmuTile* dt = (EmuTile*)(((uintptr_t)(g + nhp) + 15) & ~(uintptr_t)15);
    __nv_bfloat16* Bs = (__nv_bfloat16*)(((uintptr_t)(dt + tn.size() + tr.size()) + 255) & ~(uintptr_t)255);
    int* eb = (int*)(Bs + vs);
    std::vector<double> gh(nhp, 0.0);
    for (int i = 0; i < nh; ++i) gh[i] = -b.L * fields[i] * cabs;
    TGBA_CUDA(cudaMemcpyAsync(g, gh.data(), nhp * sizeof(double), cudaMemcpyHostToDevice, st));
    if (!tn.empty()) TGBA_CUDA(cudaMemcpyAsync(dt, tn.data(), tn.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
    if (!tr.empty())
      TGBA_CUDA(cudaMemcpyAsync(dt + tn.size(), tr.data(), tr.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemsetAsync(q0, 0, 4 * (size_t)n_un * nhp * sizeof(double), st));
    TGBA_CUDA(cudaMemsetAsync(be, 0, (size_t)m * nhp * sizeof(double), st));
    lz_start<<<nh, kRedThreads, 0, st>>>(n_un, q1);
    ++b.launches;
    double *qp = q0, *qc = q1, *qn = q2;
    for (int j = 0; j < m; ++j) {
      if (coupled) {
        if ((r = offdiag(qc, Y, nhp, Bs, eb, dt, (int)tn.size(), cn, dt + tn.size(), (int)tr.size(), cr_, 2)) != TGBA_OK) return r;
      }
      lz_step<<<nh, kRedThreads, 0, st>>>(n_un, E, g, Y, qp, qc, qn, al, be, j, m);
      ++b.launches;
      double* t = qp; qp = qc; qc = qn; qn = t;
    }
    TGBA_CUDA(cudaGetLastError());
    std::vector<double> ha((size_t)m * nhp), hb((size_t)m * nhp);
    TGBA_CUDA(cudaMemcpyAsync(ha.data(), al, ha.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaMemcpyAsync(hb.data(), be, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
    if ((r = check_status(b, st)) != TGBA_OK) return r;
    for (int i = 0; i < nh; ++i) {
      int mm = m;                                   // stop at a breakdown (an invariant subspace)
      for (int j = 1; j < m; ++j)
        if (!(std::fabs(hb[(size_t)i * m + j]) > 1e-12 * (1.0 + std::fabs(ha[(size_t)i * m])))) { mm = j; break; }
      tridiag_extremes(&ha[(size_t)i * m], &hb[(size_t)i * m], mm, &lo[i], &hi[i]);
      if (!(std::isfinite(lo[i]) && std::isfinite(hi[i]))) return fail(TGBA_ENUMERIC, "Lanczos bounds are not finite");
    }
  }
  // Gershgorin row sums of |Q| (the fallback interval)
  std::vector<double> rs;
  auto gershgorin = [&](int i, double* l, double* h) -> tgba_status {
    if (rs.empty()) {
      rs.assign(n_un, 0.0);
      if (coupled) {
        DevBuf buf(st);
        TGBA_CUDA(cudaMallocAsync(&buf.p, n_un * sizeof(double), st));
        abs_sums_ns<<<blocks_for(32 * kn_max), 256, 0, st>>>(kn_max, kr_max, Q, (double*)buf.p);
        abs_sums_r<<<blocks_for(kr_max), 256, 0, st>>>(kn_max, kr_max, Q, (double*)buf.p);
        TGBA_CUDA(cudaGetLastError());
        b.launches += 2;
        TGBA_CUDA(cudaMemcpyAsync(rs.data(), buf.p, n_un * sizeof(double), cudaMemcpyDeviceToHost, st));
        TGBA_CUDA(cudaStreamSynchronize(st));
      }
    }
    std::vector<double> eh(n_un);
    TGBA_CUDA(cudaMemcpyAsync(eh.data(), E, n_un * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
    const double ga = std::fabs(b.L * fields[i] * cabs);
    *l = 1e300; *h = -1e300;
    for (int64_t q = 0; q < n_un; ++q) {
      *l = std::min(*l, eh[q] - ga * rs[q]);
      *h = std::max(*h, eh[q] + ga * rs[q]);
    }
    return TGBA_OK;
  };
  // ---- columns: variants by decreasing kept set, Re and Im of each, padded to a tile multiple
  std::vector<int> ord(vars.size());
  for (size_t i = 0; i < vars.size(); ++i) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    return vars[x].kn != vars[y].kn ? vars[x].kn > vars[y].kn : vars[x].kr > vars[y].kr;
  });
  const int ncol = 2 * (int)vars.size();
  const int ncolp = (ncol + TC - 1) / TC * TC;
  std::vector<int64_t> out_ns(ncolp, 0), out_r(ncolp, 0), k_ns(ncolp, 0), k_r(ncolp, 0);
  for (int j = 0; j < (int)ord.size(); ++j)
    for (int h = 0; h < 2; ++h) {
      const ChebVariant& v = vars[ord[j]];
      out_ns[2 * j + h] = v.kn; k_ns[2 * j + h] = v.kr;
      out_r[2 * j + h] = v.kr; k_r[2 * j + h] = v.kn;
    }
  std::vector<EmuTile> tn = product_tiles(kn_max, ncolp, out_ns, k_ns), tr = product_tiles(kr_max, ncolp, out_r, k_r);
  const int64_t cn = emu_number_tiles(tn), cr_ = emu_number_tiles(tr);
  if (cn < 0 || cr_ < 0) return fail(TGBA_EINVAL, "quench product tiles");
  const int dt_n = n_t;
  const double dt = n_t > 1 ? t_max / (n_t - 1) : 0.0;
  cudaStream_t cap = nullptr;
  TGBA_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  struct StreamGuard { cudaStream_t s; ~StreamGuard() { if (s) cudaStreamDestroy(s); } } cap_guard{cap};
  for (int attempt = 0; attempt < 2; ++attempt) {
    // per variant: interval, terms
    std::vector<double> ec(vars.size()), R(vars.size());
    int K = 1;
    for (size_t v = 0; v < vars.size(); ++v) {
      const int i = (int)(std::find(fields.begin(), fields.end(), vars[v].hx) - fields.begin());
      double l = lo[i], h = hi[i];
      if (attempt == 1) {
        if ((r = gershgorin(i, &l, &h)) != TGBA_OK) return r;
      }
      const double half = 0.5 * (h - l);
      ec[v] = 0.5 * (h + l);
      R[v] = (attempt == 0 ? 1.02 * half + 1e-3 * (1.0 + std::fabs(ec[v])) : 1.01 * half + 1e-9) + 1e-12;
      const double xmax = R[v] * t_max;
      K = std::max(K, (int)std::ceil(xmax + 10.0 * std::cbrt(xmax) + 30.0));
    }
    const int K1 = K + 1;
    const int64_t S = n_un * ncolp;                      // one step's vectors
    const size_t vs = vec_slices(ncolp);
    const size_t tb = (tn.size() + tr.size()) * sizeof(EmuTile);
    const size_t need = sizeof(double) * ((size_t)S * K1 + S + 2 * (size_t)ncolp + 8) + ncolp * sizeof(ColPrm) + vs * 2 +
                        (size_t)ncolp * 4 + tb + 1024;
    size_t free_b = 0, tot_b = 0;
    TGBA_CUDA(cudaMemGetInfo(&free_b, &tot_b));
    if (need + ((size_t)2 << 30) > free_b)
      return fail(TGBA_ENOMEM, "the Chebyshev vectors of the batched quench need " + std::to_string(need >> 20) +
                                   " MiB of device memory");
    DevBuf vbuf(st);
    TGBA_CUDA(cudaMallocAsync(&vbuf.p, need, st));
    double* V = (double*)vbuf.p;
    double* Y = V + (size_t)S * K1;
    double* nrm = Y + S;
    ColPrm* prm = (ColPrm*)(nrm + 2 * (size_t)ncolp + 8);
    EmuTile* dtl = (EmuTile*)(((uintptr_t)(prm + ncolp) + 15) & ~(uintptr_t)15);
    __nv_bfloat16* Bs = (__nv_bfloat16*)(((uintptr_t)(dtl + tn.size() + tr.size()) + 255) & ~(uintptr_t)255);
    int* eb = (int*)(Bs + vs);
    std::vector<ColPrm> hp(ncolp, ColPrm{0.0, 0.0, 0.0, 0, 0});
    for (int j = 0; j < (int)ord.size(); ++j) {
      const int v = ord[j];
      for (int h = 0; h < 2; ++h) hp[2 * j + h] = ColPrm{-b.L * vars[v].hx * cabs, ec[v], 1.0 / R[v], vars[v].kn, vars[v].kr};
    }
    TGBA_CUDA(cudaMemcpyAsync(prm, hp.data(), ncolp * sizeof(ColPrm), cudaMemcpyHostToDevice, st));
    if (!tn.empty()) TGBA_CUDA(cudaMemcpyAsync(dtl, tn.data(), tn.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
    if (!tr.empty())
      TGBA_CUDA(cudaMemcpyAsync(dtl + tn.size(), tr.data(), tr.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemsetAsync(Y, 0, S * sizeof(double), st));
    cheb_init<<<blocks_for(S), 256, 0, st>>>(n_un, kn_max, ncolp, prm, c, V);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
    TGBA_CUDA(cudaStreamSynchronize(st));
    b.quench_prep_ms = ms_since(t_start);     // slicing of Q, Lanczos, set-up (last attempt)
    // the K steps of all variants, captured once and launched as one graph
    TGBA_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaStream_t keep = st;
    st = cap;                                            // offdiag launches on `st`
    tgba_status cr = TGBA_OK;
    const int64_t launches0 = b.launches.load();
    for (int k = 0; k < K && cr == TGBA_OK; ++k) {
      double* vk = V + (size_t)k * S;
      if (coupled)
        cr = offdiag(vk, Y, ncolp, Bs, eb, dtl, (int)tn.size(), cn, dtl + tn.size(), (int)tr.size(), cr_, 6);
      if (cr != TGBA_OK) break;
      cheb_step<<<blocks_for(S), 256, 0, cap>>>(n_un, kn_max, ncolp, E, prm, k == 0 ? 1.0 : 2.0, 1.0, Y, vk,
                                                 k == 0 ? nullptr : vk - S, vk + S);
      ++b.launches;
    }
    st = keep;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    const int64_t graph_launches = b.launches.load() - launches0;
    b.launches -= graph_launches;                        // counted when the graph runs
    if (cr != TGBA_OK) {
      if (graph) cudaGraphDestroy(graph);
      return cr;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (Chebyshev steps)");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate (Chebyshev steps)");
    struct ExecGuard { cudaGraphExec_t e; ~ExecGuard() { cudaGraphExecDestroy(e); } } exec_guard{exec};
    for (int e = 0; e < 2; ++e)
      if (b.q_ev[e] == nullptr) TGBA_CUDA(cudaEventCreate(&b.q_ev[e]));
    TGBA_CUDA(cudaEventRecord(b.q_ev[0], st));
    TGBA_CUDA(cudaGraphLaunch(exec, st));
    TGBA_CUDA(cudaEventRecord(b.q_ev[1], st));
    b.q_ev_recorded = true;
    b.launches += graph_launches;
    b.quench_flops = 0;
    for (const ChebVariant& v : vars) b.quench_flops += 8.0 * (double)K * (double)v.kn * (double)v.kr;
    // the interval check: ||v_K|| <= ||v_0|| for every column
    cheb_norms<<<ncolp, kRedThreads, 0, st>>>(n_un, V, V + (size_t)K * S, nrm);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
    {
      std::vector<double> hn(2 * (size_t)ncolp);
      TGBA_CUDA(cudaMemcpyAsync(hn.data(), nrm, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      TGBA_CUDA(cudaStreamSynchronize(st));
      if ((r = check_status(b, st)) != TGBA_OK) return r;
      bool ok = true;
      for (int q = 0; q < ncolp; ++q)
        if (!(hn[2 * q + 1] <= hn[2 * q] * (1.0 + 1e-6) + 1e-300)) ok = false;
      if (!ok) {
        if (attempt == 1) return fail(TGBA_ENUMERIC, "the Chebyshev expansion left its Gershgorin interval");
        continue;                               // redo with Gershgorin bounds
      }
    }
    // ---- moments and <sigma^x>(t), one variant at a time, with the variant's own number of
    // terms K_v <= K (the other columns' longer expansions cost it nothing): the Gram matrices
    // of its first K_v + 1 vectors and the Bessel sums over the whole time grid are tensor-core
    // FP64 products as well
    int64_t chi_max = 0;
    for (const ChebVariant& v : vars) chi_max = std::max<int64_t>(chi_max, v.kn + v.kr);
    std::vector<int> Kv(vars.size());
    for (size_t v = 0; v < vars.size(); ++v) {
      const double xmax = R[v] * t_max;
      Kv[v] = std::min(K, (int)std::ceil(xmax + 10.0 * std::cbrt(xmax) + 30.0));
    }
    const int64_t nt = std::max(1, dt_n);
    const size_t sa = std::max(emu_operand_elems(K1, (int)chi_max, TR), emu_operand_elems(K1, K1, TR));
    const size_t sb = std::max(emu_operand_elems(K1, (int)chi_max, TC), emu_operand_elems((int)nt, K1, TC));
    const size_t n_tiles_max = (size_t)((K1 + TR - 1) / TR) * (size_t)std::max<int64_t>((K1 + TC - 1) / TC, (nt + TC - 1) / TC);
    DevBuf mbuf(st);
    const size_t mdoubles = 4 * (size_t)K1 * K1 + 2 * (size_t)K1 * nt + chi_max + 8;
    TGBA_CUDA(cudaMallocAsync(&mbuf.p, mdoubles * 8 + (2 * sa + 2 * sb) * 2 + 4 * ((size_t)K1 + nt) * 4 +
                                           2 * n_tiles_max * sizeof(EmuTile) + 1024, st));
    double* Grr = (double*)mbuf.p;
    double* Gii = Grr + (size_t)K1 * K1;
    double* Gri = Gii + (size_t)K1 * K1;
    double* Gam = Gri + (size_t)K1 * K1;
    double* Ab = Gam + (size_t)K1 * K1;                   // a_k(t): [K_v + 1][t]
    double* GA = Ab + (size_t)K1 * nt;                    // Gamma a(t): column-major (K_v + 1) x n_t
    double* Ek = GA + (size_t)K1 * nt;
    double* d01 = Ek + chi_max;
    EmuTile* dtg = (EmuTile*)(((uintptr_t)(d01 + 8) + 15) & ~(uintptr_t)15);
    EmuTile* dlo = dtg + n_tiles_max;                     // the lower-triangle tiles of the Gram matrices
    __nv_bfloat16* Vr = (__nv_bfloat16*)(((uintptr_t)(dlo + n_tiles_max) + 255) & ~(uintptr_t)255);
    __nv_bfloat16* Vi = Vr + sa;
    __nv_bfloat16* Wr = Vi + sa;
    __nv_bfloat16* Wi = Wr + sb;
    int* evr = (int*)(Wi + sb);
    int* evi = evr + K1;
    int* ewr = evi + K1;
    int* ewi = ewr + (K1 > nt ? K1 : nt);
    // output tiles of a product (lower: only the tiles on or below the diagonal, for a
    // symmetric result that is read through its lower triangle; TR == TC)
    auto grid_tiles = [&](int64_t rows, int64_t cols, int64_t kdim, int64_t& n_chunks, bool lower = false) {
      std::vector<EmuTile> t;
      for (int64_t rb = 0; rb * TR < rows; ++rb)
        for (int64_t cb = 0; cb * TC < cols && (!lower || cb <= rb); ++cb)
          t.push_back(EmuTile{(int32_t)rb, (int32_t)cb, (int32_t)std::min<int64_t>(TC, r16(cols - cb * TC)),
                              (int32_t)((kdim + emu_k_block() - 1) / emu_k_block())});
      n_chunks = emu_number_tiles(t);
      return t;
    };
    for (int j = 0; j < (int)ord.size(); ++j) {
      const ChebVariant& vv = vars[ord[j]];
      const int v = ord[j];
      const int k1 = Kv[v] + 1;
      const int64_t kn = vv.kn, kr = vv.kr, chi = kn + kr;
      const double* vre = V + (size_t)(2 * j) * n_un;       // column 2j of step 0; step k at + k S
      TGBA_CUDA(cudaStreamSynchronize(st));
      const auto t_gram = clk::now();
      kept_energy<<<blocks_for(chi), 256, 0, st>>>(kn, kr, kn_max, E, Ek);
      cheb_dot01<<<1, kRedThreads, 0, st>>>(n_un, vre, vre + S, d01);
      b.launches += 2;
      int64_t cg = 0, cl = 0;
      const std::vector<EmuTile> tgv = grid_tiles(k1, k1, chi, cg), tlo = grid_tiles(k1, k1, chi, cl, true);
      if (cg < 0 || cl < 0) return fail(TGBA_EINVAL, "quench moment tiles");
      TGBA_CUDA(cudaMemcpyAsync(dtg, tgv.data(), tgv.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
      TGBA_CUDA(cudaMemcpyAsync(dlo, tlo.data(), tlo.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
      // rows k of V (K = the kept rows in their own order: kn NS rows, then kr R rows)
      const int64_t jump = kn_max - kn;
      if ((r = emu_slice(b, vre, S, 1, (int)kn, jump, nullptr, 0.0, k1, (int)chi, TR, Vr, evr, st)) != TGBA_OK) return r;
      if ((r = emu_slice(b, vre + n_un, S, 1, (int)kn, jump, nullptr, 0.0, k1, (int)chi, TR, Vi, evi, st)) != TGBA_OK)
        return r;
      if ((r = emu_slice(b, vre, S, 1, (int)kn, jump, Ek, ec[v], k1, (int)chi, TC, Wr, ewr, st)) != TGBA_OK) return r;
      if ((r = emu_slice(b, vre + n_un, S, 1, (int)kn, jump, Ek, ec[v], k1, (int)chi, TC, Wi, ewi, st)) != TGBA_OK)
        return r;
      if ((r = emu_gemm(b, Vr, evr, k1, (int)chi, Wr, ewr, k1, (int)chi, dlo, (int)tlo.size(), cl, Grr, k1, st)) != TGBA_OK)
        return r;
      if ((r = emu_gemm(b, Vi, evi, k1, (int)chi, Wi, ewi, k1, (int)chi, dlo, (int)tlo.size(), cl, Gii, k1, st)) != TGBA_OK)
        return r;
      if ((r = emu_gemm(b, Vr, evr, k1, (int)chi, Wi, ewi, k1, (int)chi, dtg, (int)tgv.size(), cg, Gri, k1, st)) != TGBA_OK)
        return r;
      cheb_gamma<<<blocks_for((int64_t)k1 * k1), 256, 0, st>>>(k1, Grr, Gii, Gri, Gam);
      ++b.launches;
      double h01 = 0.0;
      TGBA_CUDA(cudaMemcpyAsync(&h01, d01, sizeof(double), cudaMemcpyDeviceToHost, st));
      TGBA_CUDA(cudaStreamSynchronize(st));            // also: the tile list is reused below
      b.quench_gram_ms += ms_since(t_gram);
      const auto t_eval = clk::now();
      // a_k(t) for the whole grid, Gamma a(t) (Gamma symmetric: its rows are its columns), the sums
      const double scale = 1.0 / (b.L * vv.hx * vv.norm2);
      const int ms = [&] {
        int m0 = Kv[v] + 30 + (int)std::ceil(std::sqrt(40.0 * Kv[v]));
        return m0 + (m0 & 1);
      }();
      cheb_bessel<<<(int)((nt + 31) / 32), 32, 0, st>>>((int)nt, 0, dt, R[v], Kv[v], ms, Ab);
      ++b.launches;
      int64_t ct = 0;
      const std::vector<EmuTile> tt = grid_tiles(k1, nt, k1, ct);
      if (ct < 0) return fail(TGBA_EINVAL, "quench time-sum tiles");
      TGBA_CUDA(cudaMemcpyAsync(dtg, tt.data(), tt.size() * sizeof(EmuTile), cudaMemcpyHostToDevice, st));
      if ((r = emu_slice(b, Gam, k1, 1, k1, 0, nullptr, 0.0, k1, k1, TR, Vr, evr, st)) != TGBA_OK) return r;
      if ((r = emu_slice(b, Ab, 1, nt, k1, 0, nullptr, 0.0, (int)nt, k1, TC, Wr, ewi, st)) != TGBA_OK) return r;
      if ((r = emu_gemm(b, Vr, evr, k1, k1, Wr, ewi, (int)nt, k1, dtg, (int)tt.size(), ct, GA, k1, st)) != TGBA_OK) return r;
      cheb_mx<<<(int)((nt * 32 + 255) / 256), 256, 0, st>>>(k1, (int)nt, Ab, GA, R[v] * h01, scale,
                                                              mx + (int64_t)vv.out * n_t);
      ++b.launches;
      TGBA_CUDA(cudaGetLastError());
      TGBA_CUDA(cudaStreamSynchronize(st));
      b.quench_eval_ms += ms_since(t_eval);
    }
    b.quench_terms = K;
    TGBA_CUDA(cudaStreamSynchronize(st));
    return check_status(b, st);
  }
  return TGBA_OK;
}

}  // namespace tgba
