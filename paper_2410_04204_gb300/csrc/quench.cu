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
// quadratic form are kernels of this file.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
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

int blocks_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

tgba_status blas_fail(cublasStatus_t s, const char* what) {
  return fail(TGBA_ECUDA, std::string("cuBLAS ") + what + " failed with status " + std::to_string((int)s));
}

}  // namespace

void destroy_blas(void* h) { cublasDestroy((cublasHandle_t)h); }

tgba_status quench(Basis& b, int s, double h0, const double* hx, const double* ecut, int nv, double t_max, int n_t,
                   double* mx, double* norm_out, int64_t* chi_out, cudaStream_t st) {
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
    const int64_t need = 2 * L + L + 16 * (int64_t)L * L * 2 + 4 * (int64_t)L * L + 8;
    double* sc;
    tgba_status r = scratch(b, need, &sc);
    if (r != TGBA_OK) return r;
    tmp.d_theta = sc;
    tmp.d_nlab = (int*)(sc + 2 * L);
    tmp.d_work = sc + 3 * L;
    tmp.d_table = tmp.d_work + 32 * (int64_t)L * L;
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
  }
  cublasSetStream(bh, st);
  const double e_ns = b.e_ns_vac * b.J;
  for (int v = 0; v < nv; ++v) {
    std::vector<int32_t> ins, ir;
    for (int64_t q = 0; q < sec.n_ns; ++q)
      if (ecut[v] < 0 || b.ns.E[sec.ns_off + q] <= (e_ns + ecut[v]) + 1e-9) ins.push_back((int32_t)q);
    for (int64_t q = 0; q < sec.n_r; ++q)
      if (ecut[v] < 0 || b.r.E[sec.r_off + q] <= (e_ns + ecut[v]) + 1e-9) ir.push_back((int32_t)q);
    const int64_t kn = (int64_t)ins.size(), kr = (int64_t)ir.size(), n = kn + kr;
    if (chi_out) chi_out[v] = n;
    if (n == 0) return fail(TGBA_EINVAL, "a quench variant keeps no states");
    const int nb = std::min(n_t, 256);
    // scratch layout (doubles)
    const int64_t need = n * n + n + 2 * n + 2 * n + 8 + kn * kr + 3 * (2 * n * nb) + 2 * L + (kn + kr + 2) / 2 + 8;
    double* sc;
    tgba_status r = scratch(b, need, &sc);
    if (r != TGBA_OK) return r;
    double* U = sc;
    double* E = U + n * n;
    double* c = E + n;          // complex interleaved c~0
    double* a = c + 2 * n;      // [Re | Im]
    double* norm2 = a + 2 * n;
    double* Q = norm2 + 8;
    double* Y = Q + kn * kr;
    double* B = Y + 2 * n * nb;
    double* XB = B + 2 * n * nb;
    double* dth_dev = XB + 2 * n * nb;
    int32_t* idx = (int32_t*)(dth_dev + 2 * L);
    TGBA_CUDA(cudaMemcpyAsync(dth_dev, dth.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx, ins.data(), kn * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TGBA_CUDA(cudaMemcpyAsync(idx + kn, ir.data(), kr * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if ((r = build_real_heff(b, s, hx[v], U, idx, kn, idx + kn, kr, st)) != TGBA_OK) return r;
    if ((r = eig_sym(b, n, U, E, true, st)) != TGBA_OK) return r;
    TGBA_CUDA(cudaMemsetAsync(norm2, 0, sizeof(double), st));
    overlap_kernel<<<blocks_for(n), 256, 0, st>>>(kn, kr, idx, idx + kn, sec.ns_off, sec.r_off, b.d_M_ns, b.d_M_r,
                                                 b.d_modes_ns, b.d_modes_r, b.max_qp, b.d_nlab, dth_dev, base[0],
                                                 base[1], s_re, s_im, g_re, g_im, L, c, norm2);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
    // a = U~^T c~0: two real products (strided complex input)
    const double one = 1.0, zero = 0.0;
    cublasStatus_t cs = cublasDgemv(bh, CUBLAS_OP_T, (int)n, (int)n, &one, U, (int)n, c, 2, &zero, a, 1);
    if (cs == CUBLAS_STATUS_SUCCESS) cs = cublasDgemv(bh, CUBLAS_OP_T, (int)n, (int)n, &one, U, (int)n, c + 1, 2, &zero, a + n, 1);
    if (cs != CUBLAS_STATUS_SUCCESS) return blas_fail(cs, "gemv");
    if (kn > 0 && kr > 0) {
      gather_kernel<<<blocks_for(kn * kr), 256, 0, st>>>(kn, kr, idx, idx + kn, sec.n_r, b.d_P + sec.x_off, Q);
      TGBA_CUDA(cudaGetLastError());
      ++b.launches;
    }
    const double cq = cabs;
    const double dt = n_t > 1 ? t_max / (n_t - 1) : 0.0;
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
    }
    if (norm_out) TGBA_CUDA(cudaMemcpyAsync(norm_out + v, norm2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  TGBA_CUDA(cudaStreamSynchronize(st));
  return check_status(b, st);
}

}  // namespace tgba
