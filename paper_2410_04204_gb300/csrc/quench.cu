// Quench dynamics (row a9; Eq. 10, the norm statement of the Quench section, Eq. S6).
//
// Initial state Phi0 = (|0_NS(h0)> + s |0_R(h0)>)/sqrt 2, the ground states of the h_x = 0
// chain at h0, with |s| = 1 chosen so that <sigma^x>(0) = Re(s <0_NS|sigma_1|0_R>) > 0 (Fig. 2:
// the superposition of positive magnetisation).  Its overlaps with the post-quench basis follow
// Eq. S6: with D_k = theta_k(h) - theta_k(h0),
//   <phi|0_P(h0)> = prod_{0<k<pi} cos(D_k/2) * prod_{pairs (-k,k) of phi} i tan(D_k/2)
// when the momenta of phi form (-k, k) pairs (and avoid k = 0, pi), and 0 otherwise.
// Then, in the real gauge of H_eff (eigenvectors U~, eigenvalues E):
//   a = U~^T c~0,  B~(t) = U~ (e^{-iEt} a),  <sigma^x>(t) = B~^H X~ B~ / ||c0||^2,
// which is Eq. 10's B(t) = M^T e^{-iEt} M^* c0 up to the diagonal change of phase.  The two
// products per block of times are FP64 GEMMs (cuBLAS); the overlaps, phases and the final
// quadratic form are kernels of this file.  The truncated subspace is the first chi states of
// the sector in energy or in overlap order (the Quench section), and successive nested
// truncations give the convergence metric of Eq. 11.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tgba_internal.h"

namespace tgba {
namespace {

// c~0 = conj(g) c0 for the kept states (complex, interleaved), and |c0|^2 accumulated in norm2.
__global__ void overlap_kernel(int64_t kn, int64_t kr, const int32_t* __restrict__ idx_ns,
                               const int32_t* __restrict__ idx_r, int64_t ns_off, int64_t r_off,
                               const uint8_t* __restrict__ M_ns, const uint8_t* __restrict__ M_r,
                               const int16_t* __restrict__ modes_ns, const int16_t* __restrict__ modes_r, int max_qp,
                               const int* __restrict__ nlab, const double* __restrict__ dth, double base_ns,
                               double base_r, double s_re, double s_im, double g_re, double g_im, int L,
                               double* __restrict__ c, double* __restrict__ norm2) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < kn + kr; q += (int64_t)gridDim.x * blockDim.x) {
    const bool ns = q < kn;
    const int64_t st = ns ? ns_off + idx_ns[q] : r_off + idx_r[q - kn];
    const int M = ns ? M_ns[st] : M_r[st];
    const int16_t* md = (ns ? modes_ns : modes_r) + (size_t)st * max_qp;
    const int* nl = nlab + (ns ? 0 : L);
    const double* d = dth + (ns ? 0 : L);
    double mag = ns ? base_ns : base_r;
    bool paired = true;
    for (int u = 0; u < M / 2 && paired; ++u) {
      const int lo = nl[md[u]], hi = nl[md[M - 1 - u]];
      if (lo != -hi || hi <= 0 || hi == L) paired = false;
      else mag *= tan(0.5 * d[md[M - 1 - u]]);
    }
    double re = 0.0, im = 0.0;
    if (paired) {
      // value = mag * i^{M/2} (times s/sqrt2 on R, 1/sqrt2 on NS); gauge factor conj(g):
      // NS: conj(g) = i^{M/2}; R: conj(g) = (-i)^{M/2} e^{i arg C0(h)}
      const double r2 = mag * M_SQRT1_2;
      if (ns) {
        re = ((M / 2) % 2 == 0) ? r2 : -r2;      // i^{M/2} i^{M/2} = (-1)^{M/2}
      } else {
        // i^{M/2} (-i)^{M/2} = 1: value s e^{i arg C0(h)} r2
        re = r2 * (s_re * g_re - s_im * g_im);
        im = r2 * (s_re * g_im + s_im * g_re);
      }
    }
    c[2 * q] = re;
    c[2 * q + 1] = im;
    const double m2 = re * re + im * im;
    if (m2 != 0.0) atomicAdd(norm2, m2);
  }
}

// Y[:, t] = e^{-i E t} a  as [Yr | Yi] (column-major n x 2nb)
__global__ void phase_kernel(int64_t n, int nb, int t0, double dt, const double* __restrict__ E,
                             const double* __restrict__ a, double* __restrict__ Y) {
  const int64_t total = n * nb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tcol = idx / n, i = idx - tcol * n;
    const double t = dt * (double)(t0 + tcol);
    double sn, cs;
    sincos(E[i] * t, &sn, &cs);
    const double ar = a[i], ai = a[n + i];          // a stored as [Re | Im]
    Y[tcol * n + i] = ar * cs + ai * sn;             // (ar + i ai)(cs - i sn)
    Y[(nb + tcol) * n + i] = ai * cs - ar * sn;
  }
}

// mx[t] = (Br . XBr + Bi . XBi) / norm2
__global__ void quad_kernel(int64_t n, int nb, int cnt, const double* __restrict__ B, const double* __restrict__ XB,
                            const double* __restrict__ norm2, double* __restrict__ mx) {
  const int lane = threadIdx.x & 31;
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= cnt) return;
  double acc = 0.0;
  for (int64_t i = lane; i < n; i += 32)
    acc += B[(int64_t)col * n + i] * XB[(int64_t)col * n + i] + B[(int64_t)(nb + col) * n + i] * XB[(int64_t)(nb + col) * n + i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) mx[col] = acc / norm2[0];
}

// Q = P[idx_ns][idx_r] as a column-major kr x kn matrix (= transpose of the row-major block)
__global__ void gather_kernel(int64_t kn, int64_t kr, const int32_t* __restrict__ idx_ns,
                              const int32_t* __restrict__ idx_r, int64_t n_r, const double* __restrict__ P,
                              double* __restrict__ Q) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < kn * kr; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx / kr, b = idx - a * kr;
    Q[idx] = P[(int64_t)idx_ns[a] * n_r + idx_r[b]];
  }
}

// Eq. 11 at each time t: || Psi^chi(t) - Psi^chi'(t) ||^2 = sum over the larger subspace of
// |B'_a - B_a|^2 (B_a = 0 for states the smaller one lacks).  The smaller subspace's NS and R
// lists are prefixes of the larger one's (nested truncations in one ranking).  B, B': [Re | Im]
// blocks of n x n_t, column-major.  The maximum over t goes to *out (bits of a non-negative
// double, so the integer maximum is the numerical one).
__global__ void eps_kernel(int n_t, int64_t knp, int64_t krp, int64_t kn, int64_t kr, const double* __restrict__ Bp,
                           const double* __restrict__ Bc, unsigned long long* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t np = knp + krp, nc = kn + kr;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_t;
       t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int64_t i = lane; i < nc; i += 32) {
      double dre = Bc[i + t * nc], dim = Bc[i + (n_t + t) * nc];
      int64_t ip = -1;
      if (i < kn) {
        if (i < knp) ip = i;
      } else if (i - kn < krp) {
        ip = knp + (i - kn);
      }
      if (ip >= 0) {
        dre -= Bp[ip + t * np];
        dim -= Bp[ip + (n_t + t) * np];
      }
      acc = fma(dre, dre, fma(dim, dim, acc));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sqrt(acc)));
  }
}

// Z~ = G^H Z G for one parity block of sigma^x_1 sigma^x_{j+1} (Z row-major complex [k][k] over
// the kept states idx): the real-gauge phase of a state depends only on M, and for two states of
// one parity it is i^{sgn (M_a - M_b)/2} (sgn = +1 NS, -1 R).  Output: real and imaginary parts.
__global__ void zgauge_kernel(int64_t k, const int32_t* __restrict__ idx, const uint8_t* __restrict__ M, int64_t off,
                              int sgn, const double* __restrict__ Zc, double* __restrict__ Zr, double* __restrict__ Zi) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / k, c = e - a * k;
    const int p = (((sgn * ((int)M[off + idx[a]] - (int)M[off + idx[c]])) / 2) % 4 + 4) % 4;
    const double re = Zc[2 * e], im = Zc[2 * e + 1];
    double xr = re, xi = im;
    if (p == 1) { xr = -im; xi = re; }
    else if (p == 2) { xr = -re; xi = -im; }
    else if (p == 3) { xr = im; xi = -re; }
    Zr[e] = xr;
    Zi[e] = xi;
  }
}

// Connected correlator for a block of cnt times: Re(B~^H Z~ B~) / ||c0||^2 - <sigma^x>^2, with
// Y1 = Z~_re [B_re | B_im] and Y2 = Z~_im [B_re | B_im] per parity block (NS rows 0..kn-1 and R
// rows kn..n-1 of B~, stored [Re block | Im block] with leading dimension n).
__global__ void corr_kernel(int64_t n, int64_t kn, int64_t kr, int nb, int cnt, const double* __restrict__ B,
                            const double* __restrict__ Y1n, const double* __restrict__ Y2n,
                            const double* __restrict__ Y1r, const double* __restrict__ Y2r,
                            const double* __restrict__ norm2, const double* __restrict__ mx, double* __restrict__ corr) {
  const int lane = threadIdx.x & 31;
  for (int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < cnt;
       t += (int)(((int64_t)gridDim.x * blockDim.x) >> 5)) {
    double acc = 0.0;
    for (int64_t a = lane; a < kn; a += 32) {
      const double br = B[a + (int64_t)t * n], bi = B[a + (int64_t)(nb + t) * n];
      acc = fma(br, Y1n[a + (int64_t)t * kn] - Y2n[a + (int64_t)(nb + t) * kn],
                fma(bi, Y1n[a + (int64_t)(nb + t) * kn] + Y2n[a + (int64_t)t * kn], acc));
    }
    for (int64_t a = lane; a < kr; a += 32) {
      const double br = B[kn + a + (int64_t)t * n], bi = B[kn + a + (int64_t)(nb + t) * n];
      acc = fma(br, Y1r[a + (int64_t)t * kr] - Y2r[a + (int64_t)(nb + t) * kr],
                fma(bi, Y1r[a + (int64_t)(nb + t) * kr] + Y2r[a + (int64_t)t * kr], acc));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) corr[t] = acc / norm2[0] - mx[t] * mx[t];
  }
}

__global__ void gather_energy(int64_t kn, int64_t kr, const int32_t* __restrict__ idx_ns, const int32_t* __restrict__ idx_r,
                              const double* __restrict__ E_ns, const double* __restrict__ E_r, double* __restrict__ E) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kn + kr; i += (int64_t)gridDim.x * blockDim.x)
    E[i] = i < kn ? E_ns[idx_ns[i]] : E_r[idx_r[i - kn]];
}

int blocks_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

tgba_status blas_fail(cublasStatus_t s, const char* what) {
  return fail(TGBA_ECUDA, std::string("cuBLAS ") + what + " failed with status " + std::to_string((int)s));
}

}  // namespace

void destroy_blas(void* h) { cublasDestroy((cublasHandle_t)h); }

constexpr int64_t kEigenMaxStates = 4096;   // automatic method: eigendecomposition up to here

tgba_status quench(Basis& b, int s, double h0, const double* hx, const double* trunc, int nv, int order, double t_max,
                   int n_t, int method, double* mx, double* norm_out, double* eps_out, int64_t* chi_out, cudaStream_t st,
                   int j_max, double* corr_out) {
  const Sector& sec = b.sectors[s];
  const int L = b.L;
  // s = conj(z)/|z|, z = <0_NS(h0)|sigma_1|0_R(h0)>: the vacuum element of a table at h0
  Modes m0ns = make_modes(L, 0, h0 / b.J), m0r = make_modes(L, 1, h0 / b.J);
  Modes mns = make_modes(L, 0, b.h), mr = make_modes(L, 1, b.h);
  double z[2];
  {
    Basis tmp;
    tmp.L = L; tmp.device = b.device;
    std::vector<double> th(2 * L);
    std::vector<int> nl(2 * L);
    for (int i = 0; i < L; ++i) { th[i] = m0ns.theta[i]; th[L + i] = m0r.theta[i]; nl[i] = m0ns.nlab[i]; nl[L + i] = m0r.nlab[i]; }
    tmp.vac_norm = m0ns.norm * m0r.norm;
    const int64_t need = 2 * L + L + 2 * (16 * (int64_t)L * L + 4 * L + 1) + 4 * (int64_t)L * L + 8;
    double* sc;
    tgba_status r = scratch(b, need, &sc);
    if (r != TGBA_OK) return r;
    tmp.d_theta = sc;
    tmp.d_nlab = (int*)(sc + 2 * L);
    tmp.d_work = sc + 3 * L;
    tmp.d_table = tmp.d_work + 2 * (16 * (int64_t)L * L + 4 * L + 1);
    tmp.d_c0 = tmp.d_table + 4 * (int64_t)L * L;
    tmp.d_status = b.d_status;
    TGBA_CUDA(cudaMemcpyAsync(tmp.d_theta, th.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(tmp.d_nlab, nl.data(), 2 * L * sizeof(int), cudaMemcpyHostToDevice, st));
    if ((r = build_table(tmp, st)) != TGBA_OK) return r;
    TGBA_CUDA(cudaMemcpyAsync(z, tmp.d_c0, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
    if ((r = check_status(b, st)) != TGBA_OK) return r;
  }
  const double zabs = std::hypot(z[0], z[1]);
  if (!(zabs > 0)) return fail(TGBA_ENUMERIC, "vanishing vacuum element at the initial field");
  const double s_re = z[0] / zabs, s_im = -z[1] / zabs;
  const double cabs = std::hypot(b.c0_host[0], b.c0_host[1]);
  const double g_re = b.c0_host[0] / cabs, g_im = b.c0_host[1] / cabs;   // e^{i arg C0(h)}
  // Eq. S6 ingredients: D_k and prod_{0<k<pi} cos(D_k/2) per parity
  std::vector<double> dth(2 * L);
  double base[2] = {1.0, 1.0};
  for (int p = 0; p < 2; ++p) {
    const Modes& a = p ? mr : mns;
    const Modes& a0 = p ? m0r : m0ns;
    for (int i = 0; i < L; ++i) {
      dth[p * L + i] = a.theta[i] - a0.theta[i];
      if (a.nlab[i] > 0 && a.nlab[i] < L) base[p] *= std::cos(0.5 * dth[p * L + i]);
    }
  }
  cublasHandle_t bh = (cublasHandle_t)b.blas;
  if (bh == nullptr) {
    cublasStatus_t cs = cublasCreate(&bh);
    if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "create");
    b.blas = bh;
    // an explicit workspace, so that calls captured into a graph allocate nothing
    constexpr size_t kWs = 32u << 20;
    TGBA_CUDA(cudaMalloc(&b.d_blas_ws, kWs));
    cs = cublasSetWorkspace(bh, b.d_blas_ws, kWs);
    if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "workspace");
  }
  cublasSetStream(bh, st);
  const double e_ns = b.e_ns_vac * b.J;
  const double one = 1.0, zero = 0.0;
  // Ranking of the sector's states (the Quench section's construction of the truncated
  // subspace): order 0 by bare energy, order 1 by |<phi|Phi0>| (largest first), ties by energy
  // and then index.  Variant v keeps, in this ranking, the states below its cutoff (order 0) or
  // its first chi_v states (order 1); nested variants then have NS and R lists that are
  // prefixes of each other.
  const int64_t n_all = sec.n_ns + sec.n_r;
  auto energy = [&](int64_t q) { return q < sec.n_ns ? b.ns.E[sec.ns_off + q] : b.r.E[sec.r_off + q - sec.n_ns]; };
  std::vector<double> absc(n_all, 0.0);
  if (order == 1 && n_all > 0) {
    const int64_t need = 2 * n_all + 8 + 2 * L + (n_all + 2) / 2 + 8;
    double* sc;
    tgba_status r = scratch(b, need, &sc);
    if (r != TGBA_OK) return r;
    double* c = sc;
    double* norm2 = c + 2 * n_all;
    double* dth_dev = norm2 + 8;
    int32_t* idx = (int32_t*)(dth_dev + 2 * L);
    std::vector<int32_t> all(n_all);
    for (int64_t q = 0; q < sec.n_ns; ++q) all[q] = (int32_t)q;
    for (int64_t q = 0; q < sec.n_r; ++q) all[sec.n_ns + q] = (int32_t)q;
    TGBA_CUDA(cudaMemcpyAsync(dth_dev, dth.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx, all.data(), n_all * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    overlap_kernel<<<blocks_for(n_all), 256, 0, st>>>(sec.n_ns, sec.n_r, idx, idx + sec.n_ns, sec.ns_off, sec.r_off,
                                                     b.d_M_ns, b.d_M_r, b.d_modes_ns, b.d_modes_r, b.max_qp, b.d_nlab,
                                                     dth_dev, base[0], base[1], s_re, s_im, g_re, g_im, L, c, norm2);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
    std::vector<double> ch(2 * n_all);
    TGBA_CUDA(cudaMemcpyAsync(ch.data(), c, 2 * n_all * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
    for (int64_t q = 0; q < n_all; ++q) absc[q] = std::hypot(ch[2 * q], ch[2 * q + 1]);
  }
  // Sort key: |c0| quantised to 1e-10 (largest first; order 1 only), E - E_NS,vac quantised to
  // 1e-9, then (parity, M, modes): exact ties (the zero overlaps of states whose momenta are not
  // (-k, k) pairs, degenerate energies) are broken the same way whatever the rounding.
  struct Key {
    long long a, e;
    int parity, M;
    const int16_t* modes;
  };
  std::vector<Key> keys(n_all);
  for (int64_t q = 0; q < n_all; ++q) {
    const bool ns = q < sec.n_ns;
    const int64_t g = ns ? sec.ns_off + q : sec.r_off + (q - sec.n_ns);
    const int16_t* md = (ns ? b.ns.modes.data() : b.r.modes.data()) + g * b.max_qp;
    int M = 0;
    while (M < b.max_qp && md[M] >= 0) ++M;
    keys[q] = {order == 1 ? -std::llround(absc[q] * 1e10) : 0, std::llround((energy(q) - e_ns) * 1e9), ns ? 0 : 1, M, md};
  }
  std::vector<int64_t> rank(n_all);
  for (int64_t q = 0; q < n_all; ++q) rank[q] = q;
  std::sort(rank.begin(), rank.end(), [&](int64_t x, int64_t y) {
    const Key &p = keys[x], &o = keys[y];
    if (p.a != o.a) return p.a < o.a;
    if (p.e != o.e) return p.e < o.e;
    if (p.parity != o.parity) return p.parity < o.parity;
    if (p.M != o.M) return p.M < o.M;
    for (int i = 0; i < p.M; ++i)
      if (p.modes[i] != o.modes[i]) return p.modes[i] < o.modes[i];
    return x < y;
  });
  std::vector<std::vector<int32_t>> sel_ns(nv), sel_r(nv);
  int64_t n_max = 0;
  for (int v = 0; v < nv; ++v) {
    int64_t keep = n_all;
    if (order == 1) keep = std::min<int64_t>(n_all, (int64_t)trunc[v]);
    for (int64_t k = 0; k < keep; ++k) {
      const int64_t q = rank[k];
      if (order == 0 && trunc[v] >= 0 && energy(q) > (e_ns + trunc[v]) + 1e-9) break;
      if (q < sec.n_ns) sel_ns[v].push_back((int32_t)q);
      else sel_r[v].push_back((int32_t)(q - sec.n_ns));
    }
    const int64_t n = (int64_t)(sel_ns[v].size() + sel_r[v].size());
    if (n == 0) return fail(TGBA_EINVAL, "a quench variant keeps no states");
    if ((eps_out || j_max > 0) && (method == 2 || (method == 0 && n > kEigenMaxStates)))
      return fail(TGBA_EINVAL, "the convergence metric needs the eigendecomposition method (at most 4096 states "
                               "with method 0)");
    n_max = std::max(n_max, n);
  }
  double* Bbuf[2] = {nullptr, nullptr};
  if (eps_out) {
    TGBA_CUDA(cudaMemsetAsync(eps_out, 0, std::max(0, nv - 1) * sizeof(double), st));
    TGBA_CUDA(cudaMallocAsync(&Bbuf[0], 2 * sizeof(double) * (size_t)n_max * 2 * n_t, st));
    Bbuf[1] = Bbuf[0] + (size_t)n_max * 2 * n_t;
  }
  struct FreeB {
    double* p; cudaStream_t s;
    ~FreeB() { if (p) cudaFreeAsync(p, s); }
  } free_b{Bbuf[0], st};
  int64_t knp = 0, krp = 0;
  std::vector<int> cheb_vars;
  for (int v = 0; v < nv; ++v) {
    const std::vector<int32_t>& ins = sel_ns[v];
    const std::vector<int32_t>& ir = sel_r[v];
    const int64_t kn = (int64_t)ins.size(), kr = (int64_t)ir.size(), n = kn + kr;
    if (chi_out) chi_out[v] = n;
    const bool cheb = method == 2 || (method == 0 && n > kEigenMaxStates);
    if (cheb) {                                     // propagated together after this loop
      cheb_vars.push_back(v);
      continue;
    }
    double* Bcur = Bbuf[v & 1];
    double* Bprev = Bbuf[(v + 1) & 1];
    const int nb = std::min(n_t, 256);
    // scratch layout (doubles): shared part, then the eigen-path buffers
    const int64_t shared = n + 2 * n + 2 * n + 8 + kn * kr + 2 * L + (kn + kr + 2) / 2 + 8;
    const int64_t need = shared + n * n + 3 * (2 * n * nb);
    double* sc;
    tgba_status r = scratch(b, need, &sc);
    if (r != TGBA_OK) return r;
    double* E = sc;
    double* c = E + n;          // complex interleaved c~0
    double* a = c + 2 * n;      // [Re | Im]
    double* norm2 = a + 2 * n;
    double* Q = norm2 + 8;      // gathered block, column-major kr x kn (= row-major [kn][kr])
    double* dth_dev = Q + kn * kr;
    int32_t* idx = (int32_t*)(dth_dev + 2 * L);
    double* U = sc + shared;
    TGBA_CUDA(cudaMemcpyAsync(dth_dev, dth.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx, ins.data(), kn * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx + kn, ir.data(), kr * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemsetAsync(norm2, 0, sizeof(double), st));
    overlap_kernel<<<blocks_for(n), 256, 0, st>>>(kn, kr, idx, idx + kn, sec.ns_off, sec.r_off, b.d_M_ns, b.d_M_r,
                                                 b.d_modes_ns, b.d_modes_r, b.max_qp, b.d_nlab, dth_dev, base[0],
                                                 base[1], s_re, s_im, g_re, g_im, L, c, norm2);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
    if (kn > 0 && kr > 0) {
      gather_kernel<<<blocks_for(kn * kr), 256, 0, st>>>(kn, kr, idx, idx + kn, sec.n_r, b.d_P + sec.x_off, Q);
      TGBA_CUDA(cudaGetLastError());
      ++b.launches;
    }
    const double cq = cabs;
    const double dt = n_t > 1 ? t_max / (n_t - 1) : 0.0;
    cublasStatus_t cs;
    if (!cheb) {
      double* Y = U + n * n;
      double* B = Y + 2 * n * nb;
      double* XB = B + 2 * n * nb;
      if ((r = build_real_heff(b, s, hx[v], U, idx, kn, idx + kn, kr, st)) != TGBA_OK) return r;
      if ((r = eig_sym(b, n, U, E, true, st)) != TGBA_OK) return r;
      // correlators: Z~_j of the kept NS-NS and R-R blocks (reduced-form Pfaffians), before the time loop
      double* zbuf = nullptr;
      double *Zr_ns = nullptr, *Zi_ns = nullptr, *Zr_r = nullptr, *Zi_r = nullptr, *Yb = nullptr;
      struct FreeZ {
        double** p; cudaStream_t s;
        ~FreeZ() { if (*p) cudaFreeAsync(*p, s); }
      } free_z{&zbuf, st};
      if (j_max > 0) {
        const int64_t kmax = std::max(kn, kr);
        const size_t zdoubles = (size_t)j_max * 2 * (kn * kn + kr * kr) + 2 * (size_t)kmax * kmax +
                                4 * (size_t)kmax * 2 * nb + (size_t)kmax * kmax + 16;
        TGBA_CUDA(cudaMallocAsync(&zbuf, zdoubles * sizeof(double), st));
        Zr_ns = zbuf;
        Zi_ns = Zr_ns + (size_t)j_max * kn * kn;
        Zr_r = Zi_ns + (size_t)j_max * kn * kn;
        Zi_r = Zr_r + (size_t)j_max * kr * kr;
        double* Zc = Zi_r + (size_t)j_max * kr * kr;
        Yb = Zc + 2 * (size_t)kmax * kmax;
        int32_t* zp = (int32_t*)(Yb + 4 * (size_t)kmax * 2 * nb);
        for (int par = 0; par < 2; ++par) {
          const std::vector<int32_t>& lst = par ? ir : ins;
          const int64_t k = (int64_t)lst.size();
          if (k == 0) continue;
          std::vector<int32_t> hp(2 * (size_t)k * k);
          for (int64_t x = 0; x < k; ++x)
            for (int64_t y = 0; y < k; ++y) { hp[2 * (x * k + y)] = lst[x]; hp[2 * (x * k + y) + 1] = lst[y]; }
          TGBA_CUDA(cudaMemcpyAsync(zp, hp.data(), hp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
          int32_t* didx = (int32_t*)(par ? idx + kn : idx);
          // the parity's contraction table of the string up to j_max (reduced form)
          const int64_t nE = 2 * (int64_t)L + 2 * j_max;
          double* ztab = nullptr;
          TGBA_CUDA(cudaMallocAsync((void**)&ztab, (2 * nE * nE + 4) * sizeof(double), st));
          struct FreeT {
            double* p; cudaStream_t s;
            ~FreeT() { cudaFreeAsync(p, s); }
          } free_t{ztab, st};
          double* c0z = ztab + 2 * nE * nE;
          if ((r = z_table(b, par, j_max, ztab, c0z, st)) != TGBA_OK) return r;
          for (int j = 1; j <= j_max; ++j) {
            if ((r = z_reduced_elements(b, s, par, j, j_max, ztab, c0z, zp, k * k, Zc, st)) != TGBA_OK) return r;
            double* zr = (par ? Zr_r : Zr_ns) + (size_t)(j - 1) * k * k;
            double* zi = (par ? Zi_r : Zi_ns) + (size_t)(j - 1) * k * k;
            zgauge_kernel<<<blocks_for(k * k), 256, 0, st>>>(k, didx, par ? b.d_M_r : b.d_M_ns, par ? sec.r_off : sec.ns_off,
                                                             par ? -1 : 1, Zc, zr, zi);
            TGBA_CUDA(cudaGetLastError());
            ++b.launches;
          }
          TGBA_CUDA(cudaStreamSynchronize(st));      // hp is reused for the other parity
        }
      }
      // a = U~^T c~0: two real products (strided complex input)
      cs = cublasDgemv(bh, CUBLAS_OP_T, (int)n, (int)n, &one, U, (int)n, c, 2, &zero, a, 1);
      if (cs == CUBLAS_STATUS_SUCCESS) cs = cublasDgemv(bh, CUBLAS_OP_T, (int)n, (int)n, &one, U, (int)n, c + 1, 2, &zero, a + n, 1);
      if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gemv");
      for (int t0 = 0; t0 < n_t; t0 += nb) {
        const int cnt = std::min(nb, n_t - t0);
        phase_kernel<<<blocks_for(n * cnt), 256, 0, st>>>(n, nb, t0, dt, E, a, Y);
        TGBA_CUDA(cudaGetLastError());
        ++b.launches;
        cs = cublasDgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, (int)n, 2 * nb, (int)n, &one, U, (int)n, Y, (int)n, &zero, B, (int)n);
        if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gemm U Y");
        TGBA_CUDA(cudaMemsetAsync(XB, 0, 2 * n * nb * sizeof(double), st));
        if (kn > 0 && kr > 0) {
          // NS rows: cq P B_R = cq Q^T B_R ;  R rows: cq P^T B_NS = cq Q B_NS
          cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, (int)kn, 2 * nb, (int)kr, &cq, Q, (int)kr, B + kn, (int)n, &zero,
                           XB, (int)n);
          if (cs == CUBLAS_STATUS_SUCCESS)
            cs = cublasDgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, (int)kr, 2 * nb, (int)kn, &cq, Q, (int)kr, B, (int)n, &zero,
                             XB + kn, (int)n);
          if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gemm X B");
        }
        quad_kernel<<<(cnt * 32 + 255) / 256, 256, 0, st>>>(n, nb, cnt, B, XB, norm2, mx + (int64_t)v * n_t + t0);
        TGBA_CUDA(cudaGetLastError());
        ++b.launches;
        if (j_max > 0) {                              // <sigma^x_1 sigma^x_{j+1}>(t), connected
          double* Y1n = Yb;
          double* Y2n = Y1n + (size_t)std::max<int64_t>(kn, 1) * 2 * nb;
          double* Y1r = Y2n + (size_t)std::max<int64_t>(kn, 1) * 2 * nb;
          double* Y2r = Y1r + (size_t)std::max<int64_t>(kr, 1) * 2 * nb;
          for (int j = 1; j <= j_max; ++j) {
            if (kn > 0) {
              const double* zr = Zr_ns + (size_t)(j - 1) * kn * kn;
              const double* zi = Zi_ns + (size_t)(j - 1) * kn * kn;
              cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, (int)kn, 2 * nb, (int)kn, &one, zr, (int)kn, B, (int)n, &zero,
                               Y1n, (int)kn);
              if (cs == CUBLAS_STATUS_SUCCESS)
                cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, (int)kn, 2 * nb, (int)kn, &one, zi, (int)kn, B, (int)n,
                                 &zero, Y2n, (int)kn);
              if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gemm Z B (NS)");
            }
            if (kr > 0) {
              const double* zr = Zr_r + (size_t)(j - 1) * kr * kr;
              const double* zi = Zi_r + (size_t)(j - 1) * kr * kr;
              cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, (int)kr, 2 * nb, (int)kr, &one, zr, (int)kr, B + kn, (int)n,
                               &zero, Y1r, (int)kr);
              if (cs == CUBLAS_STATUS_SUCCESS)
                cs = cublasDgemm(bh, CUBLAS_OP_T, CUBLAS_OP_N, (int)kr, 2 * nb, (int)kr, &one, zi, (int)kr, B + kn,
                                 (int)n, &zero, Y2r, (int)kr);
              if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gemm Z B (R)");
            }
            corr_kernel<<<(cnt * 32 + 255) / 256, 256, 0, st>>>(n, kn, kr, nb, cnt, B, Y1n, Y2n, Y1r, Y2r, norm2,
                                                                mx + (int64_t)v * n_t + t0,
                                                                corr_out + ((int64_t)v * j_max + (j - 1)) * n_t + t0);
            TGBA_CUDA(cudaGetLastError());
            ++b.launches;
          }
        }
        if (Bcur) {                                   // keep B(t) of this variant for Eq. 11
          TGBA_CUDA(cudaMemcpyAsync(Bcur + (size_t)t0 * n, B, (size_t)n * cnt * sizeof(double), cudaMemcpyDeviceToDevice, st));
          TGBA_CUDA(cudaMemcpyAsync(Bcur + (size_t)(n_t + t0) * n, B + (size_t)n * nb, (size_t)n * cnt * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
        }
      }
      if (Bcur && v > 0) {
        eps_kernel<<<(int)std::min<int64_t>(((int64_t)n_t * 32 + 255) / 256, 152 * 8), 256, 0, st>>>(
            n_t, knp, krp, kn, kr, Bprev, Bcur, (unsigned long long*)(eps_out + v - 1));
        TGBA_CUDA(cudaGetLastError());
        ++b.launches;
      }
      knp = kn;
      krp = kr;
    }
    if (norm_out) TGBA_CUDA(cudaMemcpyAsync(norm_out + v, norm2, sizeof(double), cudaMemcpyDeviceToDevice, st));
    TGBA_CUDA(cudaStreamSynchronize(st));       // the next variant may grow the shared scratch
  }
  if (!cheb_vars.empty()) {
    // every variant keeps a prefix of the NS ranking and a prefix of the R ranking: the union
    // is the longest of each
    const std::vector<int32_t>* un_ns = &sel_ns[cheb_vars[0]];
    const std::vector<int32_t>* un_r = &sel_r[cheb_vars[0]];
    for (int v : cheb_vars) {
      if (sel_ns[v].size() > un_ns->size()) un_ns = &sel_ns[v];
      if (sel_r[v].size() > un_r->size()) un_r = &sel_r[v];
    }
    const int64_t kn = (int64_t)un_ns->size(), kr = (int64_t)un_r->size(), n = kn + kr;
    double* ub = nullptr;
    const size_t udoubles = (size_t)n + 2 * n + 8 + (size_t)kn * kr + 2 * L + (n + 2) / 2 + 8;
    TGBA_CUDA(cudaMallocAsync(&ub, udoubles * sizeof(double), st));
    struct FreeU {
      double* p; cudaStream_t s;
      ~FreeU() { cudaFreeAsync(p, s); }
    } free_u{ub, st};
    double* E = ub;
    double* c = E + n;
    double* norm2 = c + 2 * n;
    double* Q = norm2 + 8;
    double* dth_dev = Q + (size_t)kn * kr;
    int32_t* idx = (int32_t*)(dth_dev + 2 * L);
    TGBA_CUDA(cudaMemcpyAsync(dth_dev, dth.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx, un_ns->data(), kn * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx + kn, un_r->data(), kr * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemsetAsync(norm2, 0, sizeof(double), st));
    overlap_kernel<<<blocks_for(n), 256, 0, st>>>(kn, kr, idx, idx + kn, sec.ns_off, sec.r_off, b.d_M_ns, b.d_M_r,
                                                 b.d_modes_ns, b.d_modes_r, b.max_qp, b.d_nlab, dth_dev, base[0],
                                                 base[1], s_re, s_im, g_re, g_im, L, c, norm2);
    gather_energy<<<blocks_for(n), 256, 0, st>>>(kn, kr, idx, idx + kn, b.d_E_ns + sec.ns_off, b.d_E_r + sec.r_off, E);
    b.launches += 2;
    if (kn > 0 && kr > 0) {
      gather_kernel<<<blocks_for(kn * kr), 256, 0, st>>>(kn, kr, idx, idx + kn, sec.n_r, b.d_P + sec.x_off, Q);
      ++b.launches;
    }
    TGBA_CUDA(cudaGetLastError());
    // ||c0||^2 of each variant: sums of |c~0|^2 over its two prefixes
    std::vector<double> ch(2 * n), pre(n + 1, 0.0);
    TGBA_CUDA(cudaMemcpyAsync(ch.data(), c, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
    for (int64_t q = 0; q < n; ++q) pre[q + 1] = pre[q] + (ch[2 * q] * ch[2 * q] + ch[2 * q + 1] * ch[2 * q + 1]);
    std::vector<ChebVariant> cv;
    std::vector<double> norms(nv, 0.0);
    for (int v : cheb_vars) {
      ChebVariant x;
      x.out = v;
      x.kn = (int64_t)sel_ns[v].size();
      x.kr = (int64_t)sel_r[v].size();
      x.hx = hx[v];
      x.norm2 = pre[x.kn] + (pre[kn + x.kr] - pre[kn]);
      norms[v] = x.norm2;
      cv.push_back(x);
    }
    tgba_status r = quench_cheb_batch(b, Q, kn, kr, E, c, cv, t_max, n_t, mx, st);
    if (r != TGBA_OK) return r;
    if (norm_out)
      for (int v : cheb_vars) TGBA_CUDA(cudaMemcpyAsync(norm_out + v, &norms[v], sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaStreamSynchronize(st));
  }
  TGBA_CUDA(cudaStreamSynchronize(st));
  return check_status(b, st);
}

}  // namespace tgba
