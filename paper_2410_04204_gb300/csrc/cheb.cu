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
// Variants with the same kept set (differing only in h_x) form a group.  Iteration k runs,
// per group, two FP64 GEMMs on the top-left block of Q (cuBLAS) and one elementwise kernel for
// the three-term recurrence; the K iterations of all groups are captured into one CUDA graph.
#include <cublas_v2.h>

#include <algorithm>
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

// energy of row `row` of a kept set with kn NS rows (NS rows first), from the union energies
// (kn_max NS rows, then the R rows)
__device__ __forceinline__ double row_energy(const double* __restrict__ E, int64_t row, int64_t kn, int64_t kn_max) {
  return row < kn ? E[row] : E[kn_max + (row - kn)];
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

// v_0 of a group: column 2j = Re c~0, 2j + 1 = Im c~0 on the group's kept rows
__global__ void cheb_init(int64_t chi, int64_t kn, int64_t kn_max, int cols, const double* __restrict__ c,
                          double* __restrict__ V) {
  const int64_t total = chi * cols;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q % chi;
    const int col = (int)(q / chi);
    const int64_t u = row < kn ? row : kn_max + (row - kn);
    V[q] = c[2 * u + (col & 1)];
  }
}

// v_{k+1} = alpha (g Y + (E - E_c) v_k) / R - beta v_{k-1} on one group; per variant j of the
// group (columns 2j, 2j + 1): prm[3 j] = g, prm[3 j + 1] = E_c, prm[3 j + 2] = 1/R
__global__ void cheb_step(int64_t chi, int64_t kn, int64_t kn_max, int cols, const double* __restrict__ E,
                          const double* __restrict__ prm, double alpha, double beta, const double* __restrict__ Y,
                          const double* __restrict__ x, const double* __restrict__ prev, double* __restrict__ next) {
  const int64_t total = chi * cols;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q % chi;
    const int j = (int)(q / chi) >> 1;
    const double g = prm[3 * j], ec = prm[3 * j + 1], ir = prm[3 * j + 2];
    const double h = fma(g, Y[q], (row_energy(E, row, kn, kn_max) - ec) * x[q]);
    next[q] = alpha * ir * h - (prev ? beta * prev[q] : 0.0);
  }
}

// per column: ||v_0||^2 and ||v_K||^2 (one block per column)
__global__ void cheb_norms(int64_t chi, int cols, const double* __restrict__ V0, const double* __restrict__ VK,
                           double* __restrict__ out) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  double s0 = 0.0, sk = 0.0;
  for (int64_t i = threadIdx.x; i < chi; i += blockDim.x) {
    const double a = V0[(int64_t)c * chi + i], b = VK[(int64_t)c * chi + i];
    s0 = fma(a, a, s0);
    sk = fma(b, b, sk);
  }
  s0 = block_reduce(s0, sh);
  sk = block_reduce(sk, sh);
  if (threadIdx.x == 0) { out[2 * c] = s0; out[2 * c + 1] = sk; }
}

// W = (E - E_c) V for the Re and Im columns of one variant over all k: V columns at stride S
// (the k blocks of its group), W packed [re: chi x K1][im: chi x K1]
__global__ void cheb_weight(int64_t chi, int64_t kn, int64_t kn_max, int K1, int64_t S, const double* __restrict__ E,
                            double ec, const double* __restrict__ Vre, double* __restrict__ W) {
  const int64_t total = 2 * chi * K1;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q % chi;
    const int64_t k = (q / chi) % K1;
    const int part = (int)(q / (chi * K1));
    W[q] = (row_energy(E, row, kn, kn_max) - ec) * Vre[k * S + part * chi + row];
  }
}

// Re(v_0^H v_1) of one variant
__global__ void cheb_dot01(int64_t chi, int64_t S, const double* __restrict__ Vre, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < chi; i += blockDim.x)
    s = fma(Vre[i], Vre[S + i], fma(Vre[chi + i], Vre[S + chi + i], s));
  s = block_reduce(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// Gamma_kl = Re(i^{k-l} mu_kl), mu = (G_rr + G_ii) + i (G_ri - G_ri^T), G column-major K1 x K1
__global__ void cheb_gamma(int K1, const double* __restrict__ Grr, const double* __restrict__ Gii,
                           const double* __restrict__ Gri, double* __restrict__ Gam) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)K1 * K1; q += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(q / K1), k = (int)(q % K1);
    const int64_t kl = (int64_t)l * K1 + k, lk = (int64_t)k * K1 + l;
    const double re = Grr[kl] + Gii[kl], im = Gri[kl] - Gri[lk];
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
// J_0 + 2 sum J_2j = 1), one thread per time.
__global__ void cheb_bessel(int n_t, int t0, double dt, double R, int K, int m_start, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_t) return;
  const double x = R * dt * (double)(t0 + c);
  double* a = out + (int64_t)c * (K + 1);
  if (x == 0.0) {
    a[0] = 1.0;
    for (int k = 1; k <= K; ++k) a[k] = 0.0;
    return;
  }
  double jp1 = 0.0, j = 1e-300, norm = 0.0;
  for (int k = m_start; k >= 1; --k) {
    const double jm1 = (2.0 * k / x) * j - jp1;
    jp1 = j;
    j = jm1;                                   // j = J_{k-1} (unnormalised)
    if (k - 1 <= K) a[k - 1] = j;
    if ((k - 1) % 2 == 0 && k - 1 > 0) norm += 2.0 * j;
    if (fabs(j) > 1e250) {                     // rescale everything accumulated so far
      const double s = 1e-250;
      j *= s; jp1 *= s; norm *= s;
      for (int q = k - 1; q <= K && q <= m_start; ++q) a[q] *= s;
    }
  }
  norm += j;                                   // + J_0
  const double inv = 1.0 / norm;
  a[0] *= inv;
  for (int k = 1; k <= K; ++k) a[k] *= 2.0 * inv;
}

// mx[t] = (a(t)^T Gamma a(t) - e_shift) * scale, one warp per time (GA = Gamma a precomputed)
__global__ void cheb_mx(int K1, int cnt, const double* __restrict__ A, const double* __restrict__ GA, double e_shift,
                        double scale, double* __restrict__ mx) {
  const int lane = threadIdx.x & 31;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= cnt) return;
  double acc = 0.0;
  for (int k = lane; k < K1; k += 32) acc = fma(A[(int64_t)col * K1 + k], GA[(int64_t)col * K1 + k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) mx[col] = (acc - e_shift) * scale;
}

int blocks_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

tgba_status blas_fail(cublasStatus_t s, const char* what) {
  return fail(TGBA_ECUDA, std::string("cuBLAS ") + what + " failed with status " + std::to_string((int)s));
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

}  // namespace

tgba_status quench_cheb_batch(Basis& b, const double* Q, int64_t kn_max, int64_t kr_max, const double* E,
                              const double* c, const std::vector<ChebVariant>& vars, double t_max, int n_t,
                              double* mx, cudaStream_t st) {
  if (vars.empty()) return TGBA_OK;
  const int64_t n_un = kn_max + kr_max;
  const double cabs = std::hypot(b.c0_host[0], b.c0_host[1]);
  cublasHandle_t bh = (cublasHandle_t)b.blas;
  const double one = 1.0, zero = 0.0;
  cublasStatus_t cs;
  auto offdiag = [&](const double* x, int64_t ldx, double* y, int64_t ldy, int64_t kn, int64_t kr, int cols) {
    // y_NS = Q^T x_R, y_R = Q x_NS on the top-left kr x kn block of Q (ld kr_max)
    cublasStatus_t q = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, (int)kn, cols, (int)kr, &one, Q, (int)kr_max, x + kn,
                                   (int)ldx, &zero, y, (int)ldy);
    if (q == CUBLAS_STATUS_SUCCESS)
      q = cublasDgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, (int)kr, cols, (int)kn, &one, Q, (int)kr_max, x, (int)ldx, &zero,
                      y + kn, (int)ldy);
    return q;
  };
  for (const ChebVariant& v : vars)
    if (!(std::fabs(v.hx) * b.L >= 1e-3))
      return fail(TGBA_EINVAL, "the Chebyshev quench path needs |h_x| L >= 1e-3 (it reads <sigma^x> off the energy); "
                               "use method 1 for h_x = 0");
  // distinct fields: Lanczos bounds on the union of the kept states
  std::vector<double> fields;
  for (const ChebVariant& v : vars)
    if (std::find(fields.begin(), fields.end(), v.hx) == fields.end()) fields.push_back(v.hx);
  const int nh = (int)fields.size();
  std::vector<double> lo(nh), hi(nh);
  {
    const int m = (int)std::min<int64_t>(kLanczosSteps, n_un);
    DevBuf buf(st);
    const size_t doubles = (size_t)4 * n_un * nh + 2 * (size_t)m * nh + nh;
    TGBA_CUDA(cudaMallocAsync(&buf.p, doubles * sizeof(double), st));
    double* q0 = (double*)buf.p;
    double* q1 = q0 + n_un * nh;
    double* q2 = q1 + n_un * nh;
    double* Y = q2 + n_un * nh;
    double* al = Y + n_un * nh;
    double* be = al + (size_t)m * nh;
    double* g = be + (size_t)m * nh;
    std::vector<double> gh(nh);
    for (int i = 0; i < nh; ++i) gh[i] = -b.L * fields[i] * cabs;
    TGBA_CUDA(cudaMemcpyAsync(g, gh.data(), nh * sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemsetAsync(q0, 0, n_un * nh * sizeof(double), st));
    TGBA_CUDA(cudaMemsetAsync(be, 0, (size_t)m * nh * sizeof(double), st));
    lz_start<<<nh, kRedThreads, 0, st>>>(n_un, q1);
    ++b.launches;
    double *qp = q0, *qc = q1, *qn = q2;
    for (int j = 0; j < m; ++j) {
      if (kn_max > 0 && kr_max > 0) {
        if ((cs = offdiag(qc, n_un, Y, n_un, kn_max, kr_max, nh)) != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "lanczos");
      } else {
        TGBA_CUDA(cudaMemsetAsync(Y, 0, n_un * nh * sizeof(double), st));
      }
      lz_step<<<nh, kRedThreads, 0, st>>>(n_un, E, g, Y, qp, qc, qn, al, be, j, m);
      ++b.launches;
      double* t = qp; qp = qc; qc = qn; qn = t;
    }
    TGBA_CUDA(cudaGetLastError());
    std::vector<double> ha((size_t)m * nh), hb((size_t)m * nh);
    TGBA_CUDA(cudaMemcpyAsync(ha.data(), al, ha.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaMemcpyAsync(hb.data(), be, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
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
      if (kn_max > 0 && kr_max > 0) {
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
  // groups: variants with the same kept set, ordered by size
  std::vector<int> ord(vars.size());
  for (size_t i = 0; i < vars.size(); ++i) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    return vars[x].kn != vars[y].kn ? vars[x].kn < vars[y].kn : vars[x].kr < vars[y].kr;
  });
  struct Grp { int64_t kn, kr, chi; std::vector<int> members; int64_t v_off, s; };
  std::vector<Grp> groups;
  for (int i : ord) {
    if (groups.empty() || groups.back().kn != vars[i].kn || groups.back().kr != vars[i].kr)
      groups.push_back({vars[i].kn, vars[i].kr, vars[i].kn + vars[i].kr, {}, 0, 0});
    groups.back().members.push_back(i);
  }
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
        tgba_status r = gershgorin(i, &l, &h);
        if (r != TGBA_OK) return r;
      }
      const double half = 0.5 * (h - l);
      ec[v] = 0.5 * (h + l);
      R[v] = (attempt == 0 ? 1.02 * half + 1e-3 * (1.0 + std::fabs(ec[v])) : 1.01 * half + 1e-9) + 1e-12;
      const double xmax = R[v] * t_max;
      K = std::max(K, (int)std::ceil(xmax + 10.0 * std::cbrt(xmax) + 30.0));
    }
    const int K1 = K + 1;
    // storage: per group [k][column][row], columns 2j (Re), 2j + 1 (Im) of member j
    int64_t total = 0, y_max = 0, chi_max = 0, n_par = 0;
    for (Grp& g : groups) {
      g.s = g.chi * 2 * (int64_t)g.members.size();
      g.v_off = total;
      total += g.s * K1;
      y_max = std::max(y_max, g.s);
      chi_max = std::max(chi_max, g.chi);
      n_par += 3 * (int64_t)g.members.size();
    }
    const size_t need = sizeof(double) * ((size_t)total + y_max + n_par + 2 * 2 * (size_t)vars.size() + 8);
    size_t free_b = 0, tot_b = 0;
    TGBA_CUDA(cudaMemGetInfo(&free_b, &tot_b));
    if (need + ((size_t)1 << 30) > free_b)
      return fail(TGBA_ENOMEM, "the Chebyshev vectors of the batched quench need " + std::to_string(need >> 20) +
                                   " MiB of device memory");
    DevBuf vbuf(st);
    TGBA_CUDA(cudaMallocAsync(&vbuf.p, need, st));
    double* V = (double*)vbuf.p;
    double* Y = V + total;
    double* prm = Y + y_max;
    double* nrm = prm + n_par;
    std::vector<double> hp;
    for (Grp& g : groups)
      for (int i : g.members) {
        hp.push_back(-b.L * vars[i].hx * cabs);
        hp.push_back(ec[i]);
        hp.push_back(1.0 / R[i]);
      }
    TGBA_CUDA(cudaMemcpyAsync(prm, hp.data(), hp.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    // v_0, then the K steps of every group, captured once and launched as one graph
    for (Grp& g : groups)
      cheb_init<<<blocks_for(g.s), 256, 0, st>>>(g.chi, g.kn, kn_max, 2 * (int)g.members.size(), c, V + g.v_off);
    TGBA_CUDA(cudaGetLastError());
    b.launches += (int64_t)groups.size();
    TGBA_CUDA(cudaStreamSynchronize(st));
    if ((cs = cublasSetStream(bh, cap)) != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "set stream");
    TGBA_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cs = CUBLAS_STATUS_SUCCESS;
    int64_t graph_launches = 0;
    for (int k = 0; k < K && cs == CUBLAS_STATUS_SUCCESS; ++k) {
      int64_t po = 0;
      for (Grp& g : groups) {
        const int cols = 2 * (int)g.members.size();
        double* vk = V + g.v_off + (int64_t)k * g.s;
        if (g.kn > 0 && g.kr > 0) {
          cs = offdiag(vk, g.chi, Y, g.chi, g.kn, g.kr, cols);
          if (cs != CUBLAS_STATUS_SUCCESS) break;
        } else {
          cudaMemsetAsync(Y, 0, g.s * sizeof(double), cap);
        }
        cheb_step<<<blocks_for(g.s), 256, 0, cap>>>(g.chi, g.kn, kn_max, cols, E, prm + po, k == 0 ? 1.0 : 2.0, 1.0, Y,
                                                     vk, k == 0 ? nullptr : vk - g.s, vk + g.s);
        ++graph_launches;
        po += 3 * (int64_t)g.members.size();
      }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    cublasSetStream(bh, st);
    if (cs != CUBLAS_STATUS_SUCCESS) {
      if (graph) cudaGraphDestroy(graph);
      return blas_fail(cs, "chebyshev step");
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
    {
      int64_t co = 0;
      for (Grp& g : groups) {
        const int cols = 2 * (int)g.members.size();
        cheb_norms<<<cols, kRedThreads, 0, st>>>(g.chi, cols, V + g.v_off, V + g.v_off + (int64_t)K * g.s, nrm + 2 * co);
        co += cols;
      }
      TGBA_CUDA(cudaGetLastError());
      b.launches += (int64_t)groups.size();
      std::vector<double> hn(2 * co);
      TGBA_CUDA(cudaMemcpyAsync(hn.data(), nrm, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      TGBA_CUDA(cudaStreamSynchronize(st));
      bool ok = true;
      for (int64_t q = 0; q < co; ++q)
        if (!(hn[2 * q + 1] <= hn[2 * q] * (1.0 + 1e-6) + 1e-300)) ok = false;
      if (!ok) {
        if (attempt == 1) return fail(TGBA_ENUMERIC, "the Chebyshev expansion left its Gershgorin interval");
        continue;                               // redo with Gershgorin bounds
      }
    }
    // moments and <sigma^x>(t), one variant at a time
    const int nb = std::min(dt_n, 256);
    const int m_start = [&] {
      int ms = K + 30 + (int)std::ceil(std::sqrt(40.0 * K));
      return ms + (ms & 1);
    }();
    DevBuf mbuf(st);
    const size_t mdoubles = (size_t)2 * chi_max * K1 + 4 * (size_t)K1 * K1 + 2 * (size_t)K1 * nb + 8;
    TGBA_CUDA(cudaMallocAsync(&mbuf.p, mdoubles * sizeof(double), st));
    double* W = (double*)mbuf.p;
    double* Grr = W + 2 * chi_max * K1;
    double* Gii = Grr + (size_t)K1 * K1;
    double* Gri = Gii + (size_t)K1 * K1;
    double* Gam = Gri + (size_t)K1 * K1;
    double* Ab = Gam + (size_t)K1 * K1;
    double* GA = Ab + (size_t)K1 * nb;
    double* d01 = GA + (size_t)K1 * nb;
    for (Grp& g : groups)
      for (size_t j = 0; j < g.members.size(); ++j) {
        const int v = g.members[j];
        const double* vre = V + g.v_off + (int64_t)(2 * j) * g.chi;
        cheb_weight<<<blocks_for(2 * g.chi * K1), 256, 0, st>>>(g.chi, g.kn, kn_max, K1, g.s, E, ec[v], vre, W);
        cheb_dot01<<<1, kRedThreads, 0, st>>>(g.chi, g.s, vre, d01);
        const int ldv = (int)g.s;
        cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, K1, K1, (int)g.chi, &one, vre, ldv, W, (int)g.chi, &zero, Grr, K1);
        if (cs == CUBLAS_STATUS_SUCCESS)
          cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, K1, K1, (int)g.chi, &one, vre + g.chi, ldv, W + g.chi * K1,
                           (int)g.chi, &zero, Gii, K1);
        if (cs == CUBLAS_STATUS_SUCCESS)
          cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, K1, K1, (int)g.chi, &one, vre, ldv, W + g.chi * K1, (int)g.chi,
                           &zero, Gri, K1);
        if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "chebyshev moments");
        cheb_gamma<<<blocks_for((int64_t)K1 * K1), 256, 0, st>>>(K1, Grr, Gii, Gri, Gam);
        double h01 = 0.0;
        TGBA_CUDA(cudaMemcpyAsync(&h01, d01, sizeof(double), cudaMemcpyDeviceToHost, st));
        TGBA_CUDA(cudaStreamSynchronize(st));
        const double scale = 1.0 / (b.L * vars[v].hx * vars[v].norm2);
        for (int t0 = 0; t0 < dt_n; t0 += nb) {
          const int cnt = std::min(nb, dt_n - t0);
          cheb_bessel<<<(cnt + 127) / 128, 128, 0, st>>>(cnt, t0, dt, R[v], K, m_start, Ab);
          cs = cublasDgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, K1, cnt, K1, &one, Gam, K1, Ab, K1, &zero, GA, K1);
          if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gamma a");
          cheb_mx<<<(cnt * 32 + 255) / 256, 256, 0, st>>>(K1, cnt, Ab, GA, R[v] * h01, scale,
                                                          mx + (int64_t)vars[v].out * n_t + t0);
          b.launches += 2;
        }
        TGBA_CUDA(cudaGetLastError());
        b.launches += 3;
      }
    b.quench_terms = K;
    TGBA_CUDA(cudaStreamSynchronize(st));
    return TGBA_OK;
  }
  return TGBA_OK;
}

}  // namespace tgba
