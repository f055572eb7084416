// Contraction table of the Bogoliubov operators (row a3 of the hot path).
//
// For <phi_a^NS| c_1 + c_1^dag |phi_b^R> the paper writes both states as Bogoliubov operators on
// the Jordan-Wigner vacuum, so the element is the Pfaffian of the skew matrix A of pairwise
// contractions <O_a O_b> (Eq. S1-S2) over the operator string
//   [NS vacuum bra: d_k^dag, k ascending] [NS excitations: d_p, p descending] [c_1 + c_1^dag]
//   [R excitations: d_q^dag (c_pi^dag at pi), q ascending] [R vacuum: d_k, k != pi, descending]
// of which one element keeps the 2L vacuum/sigma operators F and the M + M' excitation
// operators of the two states.  Ordering the rows as [F | E] (a permutation of sign +1 for the
// kept subsets, because M and M' are even), Pf(A[F u sel]) = Pf(A_FF) Pf(S[sel, sel]) with the
// Schur complement S = A_EE + A_FE^T A_FF^{-1} A_FE.  This kernel forms A over all 4L operators
// and eliminates the F block by Parlett-Reid steps with pivoting inside F; what is left of the
// E block is S, and the product of pivots is Pf(A_FF).
//
// Diagonal gauge: with psi_a = -s_a k_a - pi/4 (s = +1 for NS bra operators, -1 for R ket
// operators), R_ab = e^{-i(psi_a + psi_b)} S_ab is real, so Pf(S[sel]) = e^{i sum psi} Pf(R[sel]);
// within a momentum sector sum s k = 0 mod 2 pi and the phase is (-i)^{n/2}.  The kernel stores R
// and records max |Im| of the rotated entries so a violation is reported, never dropped.
//
// The sums over sites j = 1..L are closed-form geometric series of plane waves.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "tgba_internal.h"

namespace tgba {
namespace {

enum { K_C = 0, K_CDAG = 1, K_D = 2, K_DDAG = 3, K_SIGMA = 4, K_MAJA = 5, K_MAJB = 6 };   // Majoranas: n = site

struct Op {
  int kind, n, pos;   // kind, momentum label (k = pi n / L), position in the operator string
  double theta;
};

struct cd { double x, y; };
__device__ __forceinline__ cd mk(double x, double y) { return cd{x, y}; }
__device__ __forceinline__ cd add(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd sub(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd mul(cd a, cd b) { return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd scal(cd a, double s) { return cd{a.x * s, a.y * s}; }
__device__ __forceinline__ double abs2(cd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cd inv(cd a) { double d = abs2(a); return cd{a.x / d, -a.y / d}; }
__device__ __forceinline__ cd expi(double t) { double s, c; sincos(t, &s, &c); return cd{c, s}; }

// Plane-wave parts of an operator: O = u sum_j e^{i su k j} c_j^dag / sqrt(L) + v sum_j e^{i sv k j} c_j / sqrt(L)
__device__ void plane(const Op& o, cd& u, int& su, cd& v, int& sv) {
  double s, c;
  sincos(0.5 * o.theta, &s, &c);
  u = mk(0, 0); v = mk(0, 0); su = 1; sv = 1;
  switch (o.kind) {
    case K_C: v = mk(1, 0); sv = -1; break;
    case K_CDAG: u = mk(1, 0); su = 1; break;
    case K_D: v = mk(s, 0); sv = -1; u = mk(0, -c); su = -1; break;      // s c_k - i c c_{-k}^dag
    case K_DDAG: u = mk(s, 0); su = 1; v = mk(0, c); sv = 1; break;      // s c_k^dag + i c c_{-k}
  }
}

// sum_{j=1}^{L} e^{i pi nq j / L}
__device__ cd geo(int nq, int L) {
  int r = ((nq % (2 * L)) + 2 * L) % (2 * L);
  if (r == 0) return mk((double)L, 0);
  if (r % 2 == 0) return mk(0, 0);
  double q = M_PI * (double)r / L;
  return mk(-1.0, cos(0.5 * q) / sin(0.5 * q));       // -1 + i cot(q/2)
}

// <0| O_a O_b |0>_c = sum_j V_a(j) U_b(j)
__device__ cd contract(const Op& a, const Op& b, int L) {
  const double rl = 1.0 / sqrt((double)L);
  if (a.kind == K_SIGMA) {            // V_a(j) = delta_{j1}: U_b(1)
    cd u, v; int su, sv;
    plane(b, u, su, v, sv);
    return scal(mul(u, expi(su * M_PI * b.n / L)), rl);
  }
  cd ua, va, ub, vb; int sua, sva, sub_, svb;
  plane(a, ua, sua, va, sva);
  if (b.kind == K_SIGMA) {            // U_b(j) = delta_{j1}: V_a(1)
    return scal(mul(va, expi(sva * M_PI * a.n / L)), rl);
  }
  plane(b, ub, sub_, vb, svb);
  cd g = geo(sva * a.n + sub_ * b.n, L);
  return scal(mul(mul(va, ub), g), 1.0 / L);
}

__device__ Op op_of(int g, int L, const int* nlab, const double* theta) {
  // nlab/theta: NS modes [0, L), R modes [L, 2L), each ascending in k
  Op o;
  if (g < L) {                                       // NS vacuum (bra): d_k^dag, ascending
    o.kind = K_DDAG; o.n = nlab[g]; o.theta = theta[g]; o.pos = g;
  } else if (g == L) {
    o.kind = K_SIGMA; o.n = 0; o.theta = 0; o.pos = 2 * L;
  } else if (g < 2 * L) {                            // R vacuum (ket): d_k, k != pi, descending
    int i = (L - 2) - (g - L - 1);
    o.kind = K_D; o.n = nlab[L + i]; o.theta = theta[L + i]; o.pos = 2 * L + g;
  } else if (g < 3 * L) {                            // NS excitations (bra): d_p, descending
    int e = g - 2 * L, i = L - 1 - e;
    o.kind = K_D; o.n = nlab[i]; o.theta = theta[i]; o.pos = L + e;
  } else {                                           // R excitations (ket), ascending
    int e = g - 2 * L, i = e - L;
    int n = nlab[L + i];
    o.kind = (n == L) ? K_CDAG : K_DDAG; o.n = n; o.theta = theta[L + i]; o.pos = L + 1 + e;
  }
  return o;
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(1024) table_kernel(int L, const int* nlab, const double* theta, double vac_norm,
                                                     cd* A, double* R, double* c0, unsigned* status) {
  const int n4 = 4 * L, n2 = 2 * L;
  __shared__ cd tau[4 * kMaxL];
  __shared__ int s_piv;
  __shared__ cd s_pf;
  // 1) A over all operators, rows/cols in the order [F | E]
  for (int idx = threadIdx.x; idx < n4 * n4; idx += blockDim.x) {
    int g = idx / n4, h = idx % n4;
    if (g > h) continue;
    cd val = mk(0, 0);
    if (g != h) {
      Op a = op_of(g, L, nlab, theta), b = op_of(h, L, nlab, theta);
      val = (a.pos < b.pos) ? contract(a, b, L) : scal(contract(b, a, L), -1.0);
    }
    A[(size_t)g * n4 + h] = val;
    A[(size_t)h * n4 + g] = scal(val, -1.0);
  }
  if (threadIdx.x == 0) s_pf = mk(1, 0);
  __syncthreads();
  // 2) Parlett-Reid on the F block, updating the whole trailing matrix
  for (int k = 0; k < n2; k += 2) {
    if (threadIdx.x < 32) {
      double best = -1; int bi = k + 1;
      for (int i = k + 1 + threadIdx.x; i < n2; i += 32) {
        double v = abs2(A[(size_t)i * n4 + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) s_piv = bi;
    }
    __syncthreads();
    const int p = s_piv, r = k + 1;
    if (p != r) {
      for (int j = threadIdx.x; j < n4; j += blockDim.x) {
        cd t = A[(size_t)r * n4 + j]; A[(size_t)r * n4 + j] = A[(size_t)p * n4 + j]; A[(size_t)p * n4 + j] = t;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        cd t = A[(size_t)i * n4 + r]; A[(size_t)i * n4 + r] = A[(size_t)i * n4 + p]; A[(size_t)i * n4 + p] = t;
      }
      __syncthreads();
    }
    const cd a = A[(size_t)k * n4 + r];
    if (threadIdx.x == 0) {
      s_pf = mul(s_pf, a);
      if (p != r) s_pf = scal(s_pf, -1.0);
    }
    const cd ia = inv(a);
    for (int j = k + 2 + threadIdx.x; j < n4; j += blockDim.x) tau[j] = mul(A[(size_t)k * n4 + j], ia);
    __syncthreads();
    const int m = n4 - (k + 2);
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = k + 2 + idx / m, j = k + 2 + idx % m;
      if (i >= j) continue;
      // A_ij += A[k+1][i] tau_j - tau_i A[k+1][j]
      cd v = add(A[(size_t)i * n4 + j], sub(mul(A[(size_t)r * n4 + i], tau[j]), mul(tau[i], A[(size_t)r * n4 + j])));
      A[(size_t)i * n4 + j] = v;
      A[(size_t)j * n4 + i] = scal(v, -1.0);
    }
    __syncthreads();
  }
  // 3) gauge rotation of the Schur complement to the real table
  for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
    int a = idx / n2, b = idx % n2;
    double val = 0;
    if (a != b) {
      cd s = A[(size_t)(n2 + a) * n4 + (n2 + b)];
      int ia = a < L ? (L - 1 - a) : (L + (a - L)), ib = b < L ? (L - 1 - b) : (L + (b - L));
      int sa = a < L ? 1 : -1, sb = b < L ? 1 : -1;
      // R = i e^{i(s_a k_a + s_b k_b)} S
      cd rot = mul(mk(0, 1), expi(M_PI * (double)(sa * nlab[ia] + sb * nlab[ib]) / L));
      cd v = mul(rot, s);
      val = v.x;
      atomic_max_pos(c0 + 2, fabs(v.y));
      atomic_max_pos(c0 + 3, fabs(v.x));
    }
    R[idx] = val;
  }
  if (threadIdx.x == 0) {
    cd pf = s_pf;
    c0[0] = pf.x * vac_norm;
    c0[1] = pf.y * vac_norm;
    if (!(abs2(pf) > 1e-200) || !isfinite(pf.x) || !isfinite(pf.y)) atomicOr(status, kStTableSingular);
  }
}

__global__ void table_check(const double* c0, unsigned* status) {
  if (!(c0[2] <= 1e-9 * c0[3])) atomicOr(status, kStTableImag);
}

// ---- the same elimination spread over the GPU: one launch per step (used by build_table)
__global__ void fill_kernel(int L, const int* nlab, const double* theta, cd* A) {
  const int n4 = 4 * L;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n4 * n4; idx += gridDim.x * blockDim.x) {
    const int g = idx / n4, h = idx % n4;
    if (g > h) continue;
    cd val = mk(0, 0);
    if (g != h) {
      Op a = op_of(g, L, nlab, theta), b = op_of(h, L, nlab, theta);
      val = (a.pos < b.pos) ? contract(a, b, L) : scal(contract(b, a, L), -1.0);
    }
    A[(size_t)g * n4 + h] = val;
    A[(size_t)h * n4 + g] = scal(val, -1.0);
  }
}

// step k: pivot inside F (rows k+1 .. 2L-1 of column k), exchange, running Pf, Gauss vector
// (n4 operators, the first n2 of them the block F that is eliminated)
__global__ void __launch_bounds__(256) pivot_kernel(int n4, int n2, int k, cd* A, cd* tau, cd* pf) {
  const int r = k + 1;
  __shared__ int s_piv;
  if (threadIdx.x < 32) {
    double best = -1; int bi = r;
    for (int i = r + threadIdx.x; i < n2; i += 32) {
      double v = abs2(A[(size_t)i * n4 + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (threadIdx.x == 0) s_piv = bi;
  }
  __syncthreads();
  const int p = s_piv;
  if (p != r) {
    for (int j = threadIdx.x; j < n4; j += blockDim.x) {
      cd t = A[(size_t)r * n4 + j]; A[(size_t)r * n4 + j] = A[(size_t)p * n4 + j]; A[(size_t)p * n4 + j] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
      cd t = A[(size_t)i * n4 + r]; A[(size_t)i * n4 + r] = A[(size_t)i * n4 + p]; A[(size_t)i * n4 + p] = t;
    }
    __syncthreads();
  }
  const cd a = A[(size_t)k * n4 + r];
  if (threadIdx.x == 0) {
    cd v = mul(*pf, a);
    *pf = (p != r) ? scal(v, -1.0) : v;
  }
  const cd ia = inv(a);
  for (int j = k + 2 + threadIdx.x; j < n4; j += blockDim.x) tau[j] = mul(A[(size_t)k * n4 + j], ia);
}

// step k: A_ij += A[k+1][i] tau_j - tau_i A[k+1][j] on the trailing upper triangle (mirrored)
__global__ void update_kernel(int n4, int k, cd* A, const cd* tau) {
  const int r = k + 1, m = n4 - (k + 2);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int i = k + 2 + idx / m, j = k + 2 + idx % m;
    if (i >= j) continue;
    cd v = add(A[(size_t)i * n4 + j], sub(mul(A[(size_t)r * n4 + i], tau[j]), mul(tau[i], A[(size_t)r * n4 + j])));
    A[(size_t)i * n4 + j] = v;
    A[(size_t)j * n4 + i] = scal(v, -1.0);
  }
}

// gauge rotation of the Schur complement to the real table, C0 and the realness record
__global__ void finalize_kernel(int L, const int* nlab, double vac_norm, const cd* A, const cd* pf, double* R,
                                double* c0, unsigned* status) {
  const int n4 = 4 * L, n2 = 2 * L;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n2 * n2; idx += gridDim.x * blockDim.x) {
    int a = idx / n2, b = idx % n2;
    double val = 0;
    if (a != b) {
      cd s = A[(size_t)(n2 + a) * n4 + (n2 + b)];
      int ia = a < L ? (L - 1 - a) : (L + (a - L)), ib = b < L ? (L - 1 - b) : (L + (b - L));
      int sa = a < L ? 1 : -1, sb = b < L ? 1 : -1;
      cd rot = mul(mk(0, 1), expi(M_PI * (double)(sa * nlab[ia] + sb * nlab[ib]) / L));
      cd v = mul(rot, s);
      val = v.x;
      atomic_max_pos(c0 + 2, fabs(v.y));
      atomic_max_pos(c0 + 3, fabs(v.x));
    }
    R[idx] = val;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const cd p = *pf;
    c0[0] = p.x * vac_norm;
    c0[1] = p.y * vac_norm;
    if (!(abs2(p) > 1e-200) || !isfinite(p.x) || !isfinite(p.y)) atomicOr(status, kStTableSingular);
  }
}

__global__ void pf_init(cd* pf) { *pf = mk(1, 0); }

// ---- the contraction table of sigma^x_1 sigma^x_{j+1} between two states of one parity
// (U(j), V(j)): the coefficients of c_j^dag and c_j in an operator at site j
__device__ void at_site(const Op& o, int j, int L, cd& U, cd& V) {
  if (o.kind == K_MAJA || o.kind == K_MAJB) {          // c_l^dag + c_l, c_l^dag - c_l
    const double on = o.n == j ? 1.0 : 0.0;
    U = mk(on, 0);
    V = mk(o.kind == K_MAJA ? on : -on, 0);
    return;
  }
  cd u, v; int su, sv;
  plane(o, u, su, v, sv);
  const double rl = 1.0 / sqrt((double)L);
  U = scal(mul(u, expi(su * M_PI * (double)o.n * j / L)), rl);
  V = scal(mul(v, expi(sv * M_PI * (double)o.n * j / L)), rl);
}

// <0| O_a O_b |0>_c = sum_j V_a(j) U_b(j), also for site-local Majoranas
__device__ cd contract_z(const Op& a, const Op& b, int L) {
  const bool ma = a.kind >= K_MAJA, mb = b.kind >= K_MAJA;
  if (!ma && !mb) return contract(a, b, L);
  cd Ua, Va, Ub, Vb;
  const int j = ma ? a.n : b.n;                         // the only site that contributes
  at_site(a, j, L, Ua, Va);
  at_site(b, j, L, Ub, Vb);
  return mul(Va, Ub);
}

// A over the listed operators (rows in list order, contractions in string order, pos)
__global__ void zfill_kernel(int n4, const Op* __restrict__ ops, int L, cd* A) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)n4 * n4;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(idx / n4), h = (int)(idx % n4);
    if (g > h) continue;
    cd val = mk(0, 0);
    if (g != h) {
      const Op a = ops[g], b = ops[h];
      val = (a.pos < b.pos) ? contract_z(a, b, L) : scal(contract_z(b, a, L), -1.0);
    }
    A[(size_t)g * n4 + h] = val;
    A[(size_t)h * n4 + g] = scal(val, -1.0);
  }
}

// S = the E block left after the elimination; c0 = norm2 Pf(A_FF)
__global__ void zextract_kernel(int n4, int n2, const cd* A, const cd* pf, double norm2, cd* S, cd* c0,
                                unsigned* status) {
  const int nE = n4 - n2;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)nE * nE;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / nE), b = (int)(idx % nE);
    S[idx] = a == b ? mk(0, 0) : A[(size_t)(n2 + a) * n4 + (n2 + b)];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const cd p = *pf;
    *c0 = scal(p, norm2);
    if (!(abs2(p) > 1e-200) || !isfinite(p.x) || !isfinite(p.y)) atomicOr(status, kStTableSingular);
  }
}

}  // namespace

// Contraction table of <phi_a| B_1 A_2 B_2 ... B_j A_{j+1} |phi_b> for two states of parity
// `parity` and j <= J.  String order: [bra vacuum: d_k^dag, k != pi, ascending] [bra
// excitations of every mode, descending: d_p (c_pi at pi)] [B_1 A_2 B_2 A_3 ... B_J A_{J+1}]
// [ket excitations, ascending: d_q^dag (c_pi^dag at pi)] [ket vacuum: d_k, k != pi,
// descending].  With F = both vacua (their block's Pfaffian is the vacuum norm, so it is well
// conditioned) and E = the rest in string order, one element is
//   Z_ab = n_P^2 Pf(A_FF) Pf(S[sel, sel]),  S = A_EE + A_FE^T A_FF^{-1} A_FE,
// with sel = (a's modes: E index L - 1 - i, i descending) ++ (the first 2j string operators:
// L .. L + 2j - 1) ++ (b's modes: L + 2J + i, ascending), an even subset, so moving the ket
// vacuum block next to the bra's costs no sign.  S: (2L + 2J)^2 complex, row-major; c0z: the
// scalar n_P^2 Pf(A_FF).
tgba_status z_table(Basis& b, int parity, int J, double* S_dev, double* c0z_dev, cudaStream_t st) {
  const int L = b.L;
  const Modes md = make_modes(L, parity, b.h);
  std::vector<Op> F1, F2, E;
  int pos = 0;
  for (int i = 0; i < L; ++i)                               // bra vacuum
    if (md.nlab[i] != L) F1.push_back({K_DDAG, md.nlab[i], pos++, md.theta[i]});
  for (int i = L - 1; i >= 0; --i) {                        // bra excitations, descending
    if (md.nlab[i] == L) E.push_back({K_C, L, pos++, 0.0});
    else E.push_back({K_D, md.nlab[i], pos++, md.theta[i]});
  }
  for (int l = 1; l <= J; ++l) {                            // the string
    E.push_back({K_MAJB, l, pos++, 0.0});
    E.push_back({K_MAJA, l + 1, pos++, 0.0});
  }
  for (int i = 0; i < L; ++i) {                             // ket excitations, ascending
    if (md.nlab[i] == L) E.push_back({K_CDAG, L, pos++, 0.0});
    else E.push_back({K_DDAG, md.nlab[i], pos++, md.theta[i]});
  }
  for (int i = L - 1; i >= 0; --i)                          // ket vacuum, descending
    if (md.nlab[i] != L) F2.push_back({K_D, md.nlab[i], pos++, md.theta[i]});
  std::vector<Op> ops(F1);
  ops.insert(ops.end(), F2.begin(), F2.end());
  ops.insert(ops.end(), E.begin(), E.end());
  const int n4 = (int)ops.size(), n2 = (int)(F1.size() + F2.size());
  // work: A (n4^2), the Gauss vector (n4), Pf(A_FF), the operator list
  const size_t work_bytes = sizeof(cd) * ((size_t)n4 * n4 + n4 + 1) + sizeof(Op) * n4 + 256;
  char* work = nullptr;
  TGBA_CUDA(cudaMallocAsync((void**)&work, work_bytes, st));
  struct FreeW {
    char* p; cudaStream_t s;
    ~FreeW() { cudaFreeAsync(p, s); }
  } free_w{work, st};
  cd* A = (cd*)work;
  cd* tau = A + (size_t)n4 * n4;
  cd* pf = tau + n4;
  Op* d_ops = (Op*)(((uintptr_t)(pf + 1) + 63) & ~(uintptr_t)63);
  TGBA_CUDA(cudaMemcpyAsync(d_ops, ops.data(), sizeof(Op) * n4, cudaMemcpyHostToDevice, st));
  int sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  auto grid = [&](int64_t work_items) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work_items + 255) / 256, (int64_t)sms * 4));
  };
  zfill_kernel<<<grid((int64_t)n4 * n4), 256, 0, st>>>(n4, d_ops, L, A);
  pf_init<<<1, 1, 0, st>>>(pf);
  for (int k = 0; k < n2; k += 2) {
    pivot_kernel<<<1, 256, 0, st>>>(n4, n2, k, A, tau, pf);
    const int64_t m = n4 - (k + 2);
    update_kernel<<<grid(m * m), 256, 0, st>>>(n4, k, A, tau);
  }
  const double nrm = parity ? b.norm_r : b.norm_ns;
  zextract_kernel<<<grid((int64_t)(n4 - n2) * (n4 - n2)), 256, 0, st>>>(n4, n2, A, pf, nrm * nrm, (cd*)S_dev,
                                                                       (cd*)c0z_dev, b.d_status);
  TGBA_CUDA(cudaGetLastError());
  b.launches += 3 + n2;
  return TGBA_OK;
}

tgba_status build_table(Basis& b, cudaStream_t st) {
  const int L = b.L, n4 = 4 * L;
  cd* A = (cd*)b.d_work;
  cd* tau = A + (size_t)n4 * n4;       // the work area holds A, the Gauss vector and Pf(A_FF)
  cd* pf = tau + n4;
  int sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  auto grid = [&](int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sms * 4)); };
  TGBA_CUDA(cudaMemsetAsync(b.d_c0, 0, 4 * sizeof(double), st));
  fill_kernel<<<grid((int64_t)n4 * n4), 256, 0, st>>>(L, b.d_nlab, b.d_theta, A);
  pf_init<<<1, 1, 0, st>>>(pf);
  for (int k = 0; k < 2 * L; k += 2) {
    pivot_kernel<<<1, 256, 0, st>>>(n4, 2 * L, k, A, tau, pf);
    const int64_t m = n4 - (k + 2);
    update_kernel<<<grid(m * m), 256, 0, st>>>(n4, k, A, tau);
  }
  finalize_kernel<<<grid((int64_t)4 * L * L), 256, 0, st>>>(L, b.d_nlab, b.vac_norm, A, pf, b.d_table, b.d_c0,
                                                           b.d_status);
  table_check<<<1, 1, 0, st>>>(b.d_c0, b.d_status);
  TGBA_CUDA(cudaGetLastError());
  b.launches += 4 + 2 * L;
  b.table_valid = true;
  return TGBA_OK;
}

}  // namespace tgba

// ------------------------------------------------------------------ allocation-free variant
// tgba_table_noalloc: the same table build for callers that must not allocate device memory
// themselves or through this library.  Examples: a process whose device memory is owned by a
// fixed-size pool that rejects outside allocations, or a latency-critical loop where the
// implicit synchronisation of cudaMalloc/cudaFree is not acceptable.  The work matrix and the
// small per-call inputs live in the file-scope arrays below instead.  They are statically
// sized for chains up to kNoAllocMaxL sites (about 1 MiB in total), and every GPU that loads
// the library keeps them until the process exits.
namespace tgba {
namespace {

constexpr int kNoAllocMaxL = 64;
constexpr int kNoAllocWork = 16 * kNoAllocMaxL * kNoAllocMaxL;   // (4L)^2 complex entries

static __device__ __align__(256) cd g_noalloc_work[kNoAllocWork];
static __device__ __align__(256) double g_noalloc_theta[2 * kNoAllocMaxL];
static __device__ __align__(256) int g_noalloc_nlab[2 * kNoAllocMaxL];
static __device__ __align__(256) double g_noalloc_c0[4];            // C0 and the realness diagnostics
static __device__ __align__(256) unsigned g_noalloc_status;

struct NoAllocPtrs {
  cd* work = nullptr;
  double* theta = nullptr;
  int* nlab = nullptr;
  double* c0 = nullptr;
  unsigned* status = nullptr;
  unsigned long long ctx = 0;   // the context the addresses belong to (0: not looked up)
};

constexpr int kMaxDevices = 64;
NoAllocPtrs g_noalloc_ptrs[kMaxDevices];
std::mutex g_noalloc_mutex;

// Identity of the current CUDA context, from the driver (cuCtxGetCurrent, cuCtxGetId: IDs are
// unique for the life of the process).  A cudaDeviceReset destroys the device's primary
// context; the next one gets a new ID, and with it the module (and its static arrays) is
// loaded again, possibly at other addresses.
tgba_status current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    TGBA_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
    TGBA_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return fail(TGBA_ECUDA, "the CUDA driver does not provide cuCtxGetCurrent/cuCtxGetId");
    get_current = (GetCurrent)f1;
    get_id = (GetId)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, id) != CUDA_SUCCESS)
    return fail(TGBA_ECUDA, "no current CUDA context");
  return TGBA_OK;
}

// Device addresses of the arrays above, looked up once per device and context (the device
// current): the host-side names of __device__ arrays are not device addresses.
tgba_status noalloc_setup(int dev, NoAllocPtrs& out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  TGBA_CUDA(cudaSetDevice(dev));               // makes the device's primary context current
  unsigned long long ctx = 0;
  tgba_status r = current_context_id(&ctx);
  if (r != TGBA_OK) return r;
  NoAllocPtrs& p = g_noalloc_ptrs[dev];
  if (p.ctx != ctx) {
    p = NoAllocPtrs{};
    NoAllocPtrs q;
    TGBA_CUDA(cudaGetSymbolAddress((void**)&q.work, g_noalloc_work));
    TGBA_CUDA(cudaGetSymbolAddress((void**)&q.theta, g_noalloc_theta));
    TGBA_CUDA(cudaGetSymbolAddress((void**)&q.nlab, g_noalloc_nlab));
    TGBA_CUDA(cudaGetSymbolAddress((void**)&q.c0, g_noalloc_c0));
    TGBA_CUDA(cudaGetSymbolAddress((void**)&q.status, g_noalloc_status));
    q.ctx = ctx;
    p = q;
  }
  out = p;
  return TGBA_OK;
}

}  // namespace
}  // namespace tgba

extern "C" tgba_status tgba_table_noalloc(int32_t L, double J, double h_z, double* table_dev, double* c0_dev,
                                          void* stream) {
  using namespace tgba;
  if (L < 4 || L % 2 || !(J > 0) || !(h_z > 0) || !std::isfinite(J) || !std::isfinite(h_z))
    return fail(TGBA_EINVAL, "need even L >= 4, J > 0 and h_z > 0");
  if (L > kNoAllocMaxL)
    return fail(TGBA_ELIMIT, "tgba_table_noalloc handles chains of at most 64 sites (its static work area); "
                             "use tgba_table for longer chains");
  if (!table_dev || !c0_dev) return fail(TGBA_EINVAL, "null output");
  int dev = 0;
  TGBA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(TGBA_ELIMIT, "device index beyond the set-up table");
  NoAllocPtrs p;
  tgba_status r = noalloc_setup(dev, p);
  if (r != TGBA_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  Modes mns = make_modes(L, 0, h_z / J), mr = make_modes(L, 1, h_z / J);
  double th[2 * kNoAllocMaxL];
  int nl[2 * kNoAllocMaxL];
  for (int i = 0; i < L; ++i) {
    th[i] = mns.theta[i]; th[L + i] = mr.theta[i];
    nl[i] = mns.nlab[i]; nl[L + i] = mr.nlab[i];
  }
  // the arrays keep the previous call's contents: clear what the kernels accumulate into
  TGBA_CUDA(cudaMemcpyAsync(p.theta, th, 2 * L * sizeof(double), cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemcpyAsync(p.nlab, nl, 2 * L * sizeof(int), cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemsetAsync(p.c0, 0, 4 * sizeof(double), st));
  TGBA_CUDA(cudaMemsetAsync(p.status, 0, sizeof(unsigned), st));
  table_kernel<<<1, 1024, 0, st>>>(L, p.nlab, p.theta, mns.norm * mr.norm, p.work, table_dev, p.c0, p.status);
  TGBA_CUDA(cudaGetLastError());
  table_check<<<1, 1, 0, st>>>(p.c0, p.status);
  TGBA_CUDA(cudaGetLastError());
  TGBA_CUDA(cudaMemcpyAsync(c0_dev, p.c0, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  unsigned w = 0;
  TGBA_CUDA(cudaMemcpyAsync(&w, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  if (w & kStTableSingular) return fail(TGBA_ENUMERIC, "the vacuum block of the contraction matrix is singular");
  if (w & kStTableImag) return fail(TGBA_ENUMERIC, "the gauge-rotated contraction table is not real");
  return TGBA_OK;
}
