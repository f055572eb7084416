// Dynamic structure factor (row a8; Eq. 8-9 and the matrix element that follows them), at k = 0
// and, through the cross-sector elements, at any momentum of the basis:
//   S(w) = 2 pi sum_a w_a L_eta(w - (E_a - E_0)),   w_a = L |<psi_0|sigma^x_1|psi_a>|^2,
//   L_eta(x) = (eta/pi) / (x^2 + eta^2).
// The weights are computed in FP64 in the real gauge (w_a = L (u_a^T X~ u_0)^2 with X~ the
// real-gauge <phi|sigma^x_1|phi'>), then the Lorentzian sum runs in FP32 with FP32
// accumulation.  To keep the FP32 sum accurate near the peaks, w_i and E_a - E_0 are each
// carried as an unevaluated float pair (hi + lo), and x = (w_hi - e_hi) + (w_lo - e_lo): the
// first difference is exact when the two are within a factor of two (Sterbenz), which is where
// the Lorentzian is largest.  Each lane sums a strided share of the states, then a warp-shuffle
// tree adds the 32 partial sums.
#include <algorithm>

#include "tgba_internal.h"

namespace tgba {
namespace {

// Products with a real-gauge sigma^x_1 block c P (c = |C0|, P [rows][cols] row-major):
//   sigma_rows: out[i] = c sum_j P[i][j] x[j]   (a warp per row, coalesced along the row)
//   sigma_cols: out[j] = c sum_i P[i][j] x[i]   (a thread per column, coalesced across the warp)
__global__ void sigma_rows(int64_t rows, int64_t cols, const double* __restrict__ P, const double* __restrict__ x,
                           const double* __restrict__ c0, double* __restrict__ out) {
  const double c = sqrt(c0[0] * c0[0] + c0[1] * c0[1]);
  const int lane = threadIdx.x & 31;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < rows;
       a += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int64_t b = lane; b < cols; b += 32) acc = fma(P[a * cols + b], x[b], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[a] = c * acc;
  }
}

__global__ void sigma_cols(int64_t rows, int64_t cols, const double* __restrict__ P, const double* __restrict__ x,
                           const double* __restrict__ c0, double* __restrict__ out) {
  const double c = sqrt(c0[0] * c0[0] + c0[1] * c0[1]);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < cols; b += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t a = 0; a < rows; ++a) acc = fma(P[a * cols + b], x[a], acc);
    out[b] = c * acc;
  }
}

// w_a = L (sum_i U[i][a] v_i)^2, dE_a = E_a - E_ref[0], and the float pairs of the FP32 stage.
__global__ void weights_kernel(int64_t n, const double* __restrict__ U, const double* __restrict__ v,
                               const double* __restrict__ E, const double* __restrict__ E_ref, double L,
                               double two_eta, double* __restrict__ w, double* __restrict__ dE,
                               float* __restrict__ e_hi, float* __restrict__ e_lo, float* __restrict__ cw) {
  const int lane = threadIdx.x & 31;
  const double e0 = E_ref[0];
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n;
       a += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int64_t i = lane; i < n; i += 32) acc = fma(U[a * n + i], v[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double wa = L * acc * acc, d = E[a] - e0;
      w[a] = wa;
      dE[a] = d;
      const float hi = (float)d;
      e_hi[a] = hi;
      e_lo[a] = (float)(d - (double)hi);
      cw[a] = (float)(two_eta * wa);      // 2 pi * (eta / pi) * w_a
    }
  }
}

constexpr int kWPerWarp = 4;

__global__ void lorentz_kernel(int n_w, double w_min, double w_span, int64_t n, const float* __restrict__ e_hi,
                               const float* __restrict__ e_lo, const float* __restrict__ cw, float eta2,
                               float* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int i0 = warp * kWPerWarp;
  if (i0 >= n_w) return;
  float wh[kWPerWarp], wl[kWPerWarp], acc[kWPerWarp];
#pragma unroll
  for (int q = 0; q < kWPerWarp; ++q) {
    const int i = min(i0 + q, n_w - 1);
    const double w = n_w > 1 ? w_min + (w_span * i) / (n_w - 1) : w_min;
    wh[q] = (float)w;
    wl[q] = (float)(w - (double)wh[q]);
    acc[q] = 0.0f;
  }
  for (int64_t a = lane; a < n; a += 32) {
    const float eh = e_hi[a], el = e_lo[a], c = cw[a];
#pragma unroll
    for (int q = 0; q < kWPerWarp; ++q) {
      const float x = (wh[q] - eh) + (wl[q] - el);
      acc[q] += c / fmaf(x, x, eta2);
    }
  }
#pragma unroll
  for (int q = 0; q < kWPerWarp; ++q) {
    float s = acc[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && i0 + q < n_w) S[i0 + q] = s;
  }
}

}  // namespace

tgba_status dsf(Basis& b, int s, double h_x, double w_min, double w_max, int n_w, double eta, float* S,
                double* evals, int n_ev, double* weights, double* dE, cudaStream_t st) {
  const Sector& sec = b.sectors[s];
  const int64_t n = sec.n_ns + sec.n_r;
  if (n == 0) return fail(TGBA_EINVAL, "empty sector");
  // scratch: A (n x n), E (n), v (n), w (n), dE (n), 3 float arrays (n)
  const int64_t need = n * n + 5 * n + (3 * n + 1) / 2 + 8;
  if (need > b.eig_a_cap) {
    if (b.d_eig_a) cudaFree(b.d_eig_a);
    b.d_eig_a = nullptr;
    b.eig_a_cap = 0;
    if (cudaMalloc(&b.d_eig_a, need * sizeof(double)) != cudaSuccess) return fail(TGBA_ENOMEM, "DSF scratch");
    b.eig_a_cap = need;
  }
  double* A = b.d_eig_a;
  double* E = A + n * n;
  double* v = E + n;
  double* w = v + n;
  double* d = w + n;
  float* e_hi = (float*)(d + n);
  float* e_lo = e_hi + n;
  float* cw = e_lo + n;
  tgba_status r = build_real_heff(b, s, h_x, A, nullptr, sec.n_ns, nullptr, sec.n_r, st);
  if (r != TGBA_OK) return r;
  if ((r = eig_sym(b, n, A, E, true, st)) != TGBA_OK) return r;
  const double* P = b.d_P + sec.x_off;
  // v = X~ u0, u0 = the first column of A:  v_ns = c P u0_r,  v_r = c P^T u0_ns
  if (sec.n_ns > 0 && sec.n_r > 0) {
    sigma_rows<<<(int)std::min<int64_t>((sec.n_ns * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
        sec.n_ns, sec.n_r, P, A + sec.n_ns, b.d_c0, v);
    sigma_cols<<<(int)std::min<int64_t>((sec.n_r + 255) / 256, 152 * 16), 256, 0, st>>>(sec.n_ns, sec.n_r, P, A,
                                                                                       b.d_c0, v + sec.n_ns);
    b.launches += 2;
  } else {
    TGBA_CUDA(cudaMemsetAsync(v, 0, n * sizeof(double), st));
  }
  weights_kernel<<<(int)std::min<int64_t>((n * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
      n, A, v, E, E, (double)b.L, 2.0 * eta, w, d, e_hi, e_lo, cw);
  const int warps = (n_w + kWPerWarp - 1) / kWPerWarp;
  lorentz_kernel<<<(warps * 32 + 255) / 256, 256, 0, st>>>(n_w, w_min, w_max - w_min, n, e_hi, e_lo, cw,
                                                          (float)(eta * eta), S);
  TGBA_CUDA(cudaGetLastError());
  b.launches += 2;
  if (evals && n_ev > 0)
    TGBA_CUDA(cudaMemcpyAsync(evals, E, std::min<int64_t>(n_ev, n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (weights) TGBA_CUDA(cudaMemcpyAsync(weights, w, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (dE) TGBA_CUDA(cudaMemcpyAsync(dE, d, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return check_status(b, st);
}

// S(k, w) at the momentum k of sector s (Eq. 8-9 with the matrix element that follows them:
// <psi_a^k|sigma^x_k|psi_0> = sqrt(L) e^{-ik} <psi_a^k|sigma^x_1|psi_0>):
//   w_a = L (u_a^T Y~ u_0)^2,  Y~ = c [[0, P(NS_k, R_0)], [P(NS_0, R_k)^T, 0]],
// with u_0 the ground state of the K = 0 sector s0 and u_a the eigenvectors of sector s, all in
// the real gauge (the gauge depends only on a state's parity and M, so the cross-sector block
// is real like the diagonal ones).  The cross blocks P are Pfaffians of the same contraction
// table, for pairs whose two states lie in different sectors.
tgba_status dsf_k(Basis& b, int s, int s0, double h_x, double w_min, double w_max, int n_w, double eta, float* S,
                  double* evals, int n_ev, double* weights, double* dE, cudaStream_t st) {
  const Sector& sk = b.sectors[s];
  const Sector& sz = b.sectors[s0];
  const int64_t nk = sk.n_ns + sk.n_r, n0 = sz.n_ns + sz.n_r;
  if (nk == 0 || n0 == 0) return fail(TGBA_EINVAL, "empty sector");
  const bool same = s == s0;
  const int64_t need = n0 * n0 + n0 + (same ? 0 : nk * nk + nk) + sk.n_ns * sz.n_r + sz.n_ns * sk.n_r + 3 * nk +
                       (3 * nk + 1) / 2 + 64;
  double* A0;
  tgba_status r = scratch(b, need, &A0);
  if (r != TGBA_OK) return r;
  double* E0 = A0 + n0 * n0;
  double* Ak = same ? A0 : E0 + n0;
  double* Ek = same ? E0 : Ak + nk * nk;
  double* P1 = Ek + nk;                   // [n_ns(s)][n_r(s0)]
  double* P2 = P1 + sk.n_ns * sz.n_r;     // [n_ns(s0)][n_r(s)]
  double* v = P2 + sz.n_ns * sk.n_r;
  double* w = v + nk;
  double* d = w + nk;
  float* e_hi = (float*)(d + nk);
  float* e_lo = e_hi + nk;
  float* cw = e_lo + nk;
  if ((r = build_real_heff(b, s0, h_x, A0, nullptr, sz.n_ns, nullptr, sz.n_r, st)) != TGBA_OK) return r;
  if ((r = eig_sym(b, n0, A0, E0, true, st)) != TGBA_OK) return r;
  if (!same) {
    if ((r = build_real_heff(b, s, h_x, Ak, nullptr, sk.n_ns, nullptr, sk.n_r, st)) != TGBA_OK) return r;
    if ((r = eig_sym(b, nk, Ak, Ek, true, st)) != TGBA_OK) return r;
  }
  if ((r = run_pfaffian_cross(b, s, s0, P1, st)) != TGBA_OK) return r;
  if ((r = run_pfaffian_cross(b, s0, s, P2, st)) != TGBA_OK) return r;
  // v = Y~ u0:  v_ns(k) = c P1 u0_r,  v_r(k) = c P2^T u0_ns
  TGBA_CUDA(cudaMemsetAsync(v, 0, nk * sizeof(double), st));
  if (sk.n_ns > 0 && sz.n_r > 0) {
    sigma_rows<<<(int)std::min<int64_t>((sk.n_ns * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
        sk.n_ns, sz.n_r, P1, A0 + sz.n_ns, b.d_c0, v);
    ++b.launches;
  }
  if (sz.n_ns > 0 && sk.n_r > 0) {
    sigma_cols<<<(int)std::min<int64_t>((sk.n_r + 255) / 256, 152 * 16), 256, 0, st>>>(sz.n_ns, sk.n_r, P2, A0,
                                                                                      b.d_c0, v + sk.n_ns);
    ++b.launches;
  }
  weights_kernel<<<(int)std::min<int64_t>((nk * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
      nk, Ak, v, Ek, E0, (double)b.L, 2.0 * eta, w, d, e_hi, e_lo, cw);
  const int warps = (n_w + kWPerWarp - 1) / kWPerWarp;
  lorentz_kernel<<<(warps * 32 + 255) / 256, 256, 0, st>>>(n_w, w_min, w_max - w_min, nk, e_hi, e_lo, cw,
                                                          (float)(eta * eta), S);
  TGBA_CUDA(cudaGetLastError());
  b.launches += 2;
  if (evals && n_ev > 0)
    TGBA_CUDA(cudaMemcpyAsync(evals, Ek, std::min<int64_t>(n_ev, nk) * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (weights) TGBA_CUDA(cudaMemcpyAsync(weights, w, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (dE) TGBA_CUDA(cudaMemcpyAsync(dE, d, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return check_status(b, st);
}

}  // namespace tgba
