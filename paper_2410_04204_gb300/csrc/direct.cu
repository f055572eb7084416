// The paper-literal evaluation of X (Appendix A, Eq. S1-S2), one CTA per element: both states
// are products of Bogoliubov operators on the Jordan-Wigner vacuum (Eq. S3), so
//   X_ab = <phi_a^NS| (c_1 + c_1^dag) |phi_b^R> = n_NS n_R Pf(A),   A_uv = <0|o_u o_v|0>  (u < v),
// over the string of m = 2L + M_a + M_b linear operators o = sum_j (U_j c_j^dag + V_j c_j):
//   d_k^dag for every NS mode, k ascending          (the bra <0|_NS)
//   d_p for p in phi_a, descending                  (the bra's excitations)
//   c_1 + c_1^dag                                   (sigma^x_1 after the Jordan-Wigner map)
//   d_q^dag for q in phi_b, ascending (c_pi^dag at pi)  (the ket's excitations)
//   d_k for every R mode k != pi, descending        (the ket |0>_R)
// with d_k = sin(theta_k/2) c_k - i cos(theta_k/2) c_{-k}^dag, c_k = L^{-1/2} sum_j e^{-ikj} c_j,
// and <0|c_j c_l^dag|0> = delta_jl, so A_uv = sum_j V_u(j) U_v(j).  The Pfaffian is a complex
// Parlett-Reid elimination with partial pivoting in shared memory (packed strict upper
// triangle), the CTA's threads sharing each step's pivot search, exchange and rank-2 update.
// This is the O(m^3)-per-element form the paper describes; the production path evaluates the
// same numbers through the contraction table (reduced form, pfaffian.cu), and this kernel
// checks it on the GPU.  The same kernel gives the elements of sigma^x_1 sigma^x_{j+1} between
// two states of one parity (the equal-time correlators after a quench): after the
// Jordan-Wigner map, with A_l = c_l^dag + c_l and B_l = c_l^dag - c_l (1 - 2 n_l = A_l B_l),
// sigma^x_1 sigma^x_{j+1} = B_1 A_2 B_2 ... B_j A_{j+1}, a string of 2j Majoranas that takes the
// place of sigma^x_1, between vacua of the same parity.  z_reduced_kernel evaluates those
// elements from the contraction table of z_table instead (the vacua contracted once): a
// Pfaffian of size M_a + 2j + M_b per element, which reaches chains the direct string does not.
#include <cuComplex.h>

#include <algorithm>

#include "tgba_internal.h"

namespace tgba {
namespace {

constexpr int kDirThreads = 128;

__device__ __forceinline__ int pk(int i, int j, int m) { return i * m - ((i * (i + 1)) >> 1) + (j - i - 1); }

// entry (i, j) of the skew matrix held as its packed strict upper triangle T
__device__ __forceinline__ double2 get(const double2* T, int i, int j, int m) {
  if (i < j) return T[pk(i, j, m)];
  const double2 v = T[pk(j, i, m)];
  return make_double2(-v.x, -v.y);
}
__device__ __forceinline__ void set(double2* T, int i, int j, int m, double2 v) {
  if (i < j) T[pk(i, j, m)] = v;
  else T[pk(j, i, m)] = make_double2(-v.x, -v.y);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// Pfaffian of the m x m skew matrix held as its packed strict upper triangle T (destroyed):
// complex Parlett-Reid with partial pivoting, two indices per step, the CTA's kDirThreads
// threads sharing each step's pivot search, exchange and rank-2 update.  Every thread of the
// CTA calls it and gets the result.  rowR, tau: m entries of scratch.
__device__ double2 pf_packed(double2* T, int m, double2* rowR, double2* tau) {
  __shared__ double red_v[kDirThreads];
  __shared__ int red_i[kDirThreads];
  __shared__ double2 piv;
  __shared__ int zero_col;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = kDirThreads / 32;
  double2 pf = make_double2(1.0, 0.0);
  for (int k = 0; k + 1 < m; k += 2) {
    // pivot: the largest |A[k][x]|, x > k (ties: the smallest x)
    double best = -1.0;
    int bi = k + 1;
    for (int x = k + 1 + threadIdx.x; x < m; x += kDirThreads) {
      const double2 v = T[pk(k, x, m)];
      const double a2 = fma(v.x, v.x, v.y * v.y);
      if (a2 > best) { best = a2; bi = x; }
    }
    red_v[threadIdx.x] = best;
    red_i[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int t = 1; t < kDirThreads; ++t)
        if (red_v[t] > best || (red_v[t] == best && red_i[t] < bi)) { best = red_v[t]; bi = red_i[t]; }
      red_i[0] = bi;
      zero_col = !(best > 0.0);
    }
    __syncthreads();
    if (zero_col) { pf = make_double2(0.0, 0.0); break; }       // block-uniform
    const int R = k + 1, C = red_i[0];
    if (C != R) {                                   // exchange indices R and C
      for (int x = threadIdx.x; x < m; x += kDirThreads) {
        if (x == R || x == C) continue;
        const double2 a = get(T, R, x, m), b = get(T, C, x, m);
        set(T, R, x, m, b);
        set(T, C, x, m, a);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double2 v = T[pk(R, C, m)];
        T[pk(R, C, m)] = make_double2(-v.x, -v.y);
      }
      pf = make_double2(-pf.x, -pf.y);
      __syncthreads();
    }
    if (threadIdx.x == 0) piv = T[pk(k, R, m)];
    __syncthreads();
    const double2 a = piv;
    pf = cmul(pf, a);
    const double den = fma(a.x, a.x, a.y * a.y);
    const double2 ia = make_double2(a.x / den, -a.y / den);
    for (int x = k + 2 + threadIdx.x; x < m; x += kDirThreads) {
      tau[x] = cmul(T[pk(k, x, m)], ia);            // Gauss vector
      rowR[x] = T[pk(R, x, m)];
    }
    __syncthreads();
    // A_ij += A_Ri tau_j - tau_i A_Rj  for k + 2 <= i < j
    for (int gi = k + 2 + warp; gi < m; gi += nwarp) {
      const double2 ri = rowR[gi], ti = tau[gi];
      double2* rowp = T + pk(gi, gi + 1, m) - (gi + 1);   // rowp[gj] = A[gi][gj]
      for (int gj = gi + 1 + lane; gj < m; gj += 32) {
        double2 w = rowp[gj];
        const double2 p1 = cmul(ri, tau[gj]), p2 = cmul(ti, rowR[gj]);
        w.x += p1.x - p2.x;
        w.y += p1.y - p2.y;
        rowp[gj] = w;
      }
    }
    __syncthreads();
  }
  return pf;
}

// One operator of the string, o = sum_j (U(j) c_j^dag + V(j) c_j) with U = a phi and V = b phi
// for a common site function phi: phi(j) = e^{i pi ph j / L} / sqrt(L) for a mode operator
// (loc = 0), phi(j) = delta_{j, loc} for a site operator (loc >= 1).  Then Eq. S2's
// A_uv = sum_j V_u(j) U_v(j) = b_u a_v sum_j phi_u(j) phi_v(j), and the site sum takes one of
// three forms: G(ph_u + ph_v) = (1/L) sum_{j=1..L} e^{i pi (ph_u + ph_v) j / L} (two mode
// operators, tabulated once per CTA by summing over the sites), phi_mode(loc) (a mode and a
// site operator), delta_{loc_u, loc_v} (two site operators).
struct DirOp {
  double2 a, b;
  int ph, loc;
};

__device__ __forceinline__ int wrap2L(int x, int L) {
  const int m = 2 * L;
  x %= m;
  return x < 0 ? x + m : x;
}

// Pfaffian of the m x m skew matrix held as its packed strict upper triangle T (destroyed), by
// one warp: complex Parlett-Reid with partial pivoting, two indices per step, the pivot search
// by shuffles and only warp barriers.  The rank-2 update walks rows i and m - 1 - (i - k - 2)
// together (lengths adding up to m - k - 3), so the lanes stay busy on the short rows.  Every
// lane gets the result.  rowR, tau: m entries of the warp's scratch.
__device__ double2 pf_packed_warp(double2* T, int m, double2* rowR, double2* tau, int lane) {
  double2 pf = make_double2(1.0, 0.0);
  for (int k = 0; k + 1 < m; k += 2) {
    double best = -1.0;
    int bi = k + 1;
    for (int x = k + 1 + lane; x < m; x += 32) {
      const double2 v = T[pk(k, x, m)];
      const double a2 = fma(v.x, v.x, v.y * v.y);
      if (a2 > best) { best = a2; bi = x; }
    }
    for (int o = 16; o > 0; o >>= 1) {                 // argmax, ties: the smallest index
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > 0.0)) { pf = make_double2(0.0, 0.0); break; }    // warp-uniform
    const int R = k + 1, C = bi;
    if (C != R) {                                      // exchange indices R and C
      for (int x = lane; x < m; x += 32) {
        if (x == R || x == C) continue;
        const double2 a = get(T, R, x, m), b = get(T, C, x, m);
        set(T, R, x, m, b);
        set(T, C, x, m, a);
      }
      __syncwarp();
      if (lane == 0) {
        const double2 v = T[pk(R, C, m)];
        T[pk(R, C, m)] = make_double2(-v.x, -v.y);
      }
      pf = make_double2(-pf.x, -pf.y);
      __syncwarp();
    }
    const double2 a = T[pk(k, R, m)];
    pf = cmul(pf, a);
    const double den = fma(a.x, a.x, a.y * a.y);
    const double2 ia = make_double2(a.x / den, -a.y / den);
    for (int x = k + 2 + lane; x < m; x += 32) {
      tau[x] = cmul(T[pk(k, x, m)], ia);               // Gauss vector
      rowR[x] = T[pk(R, x, m)];
    }
    __syncwarp();
    // A_ij += A_Ri tau_j - tau_i A_Rj  for k + 2 <= i < j: eight FMAs per complex entry
    const int span = m - k - 3;                        // entries of rows i1 and i2 together
    for (int t = 0; 2 * t <= span; ++t) {
      const int i1 = k + 2 + t, i2 = m - 1 - t;
      const int len1 = m - 1 - i1, len2 = (i2 > i1) ? m - 1 - i2 : 0;
      for (int p = lane; p < len1 + len2; p += 32) {
        const int gi = p < len1 ? i1 : i2;
        const int gj = gi + 1 + (p < len1 ? p : p - len1);
        const double2 ri = rowR[gi], ti = tau[gi], rj = rowR[gj], tj = tau[gj];
        double2* w = T + pk(gi, gj, m);
        double2 v = *w;
        v.x = fma(ri.x, tj.x, v.x);
        v.x = fma(-ri.y, tj.y, v.x);
        v.x = fma(-ti.x, rj.x, v.x);
        v.x = fma(ti.y, rj.y, v.x);
        v.y = fma(ri.x, tj.y, v.y);
        v.y = fma(ri.y, tj.x, v.y);
        v.y = fma(-ti.x, rj.y, v.y);
        v.y = fma(-ti.y, rj.x, v.y);
        *w = v;
      }
    }
    __syncwarp();
  }
  return pf;
}

// One warp per element (a CTA holds `wpc` warps, each with its own string and packed triangle
// in shared memory); the site tables W (e^{i pi n / L}, n mod 2L) and G are built once per CTA.
__global__ void x_direct_kernel(const int32_t* __restrict__ pairs, int64_t n_pairs, int pa_par, int pb_par, int jmid,
                                int64_t a_off, int64_t b_off, int64_t n_a, int64_t n_b, int L,
                                const double* __restrict__ theta, const int* __restrict__ nlab,
                                const int16_t* __restrict__ modes_ns, const int16_t* __restrict__ modes_r, int max_qp,
                                double vac_norm, int wpc, double* __restrict__ out, unsigned* __restrict__ status) {
  extern __shared__ double smem_d[];
  const int mmax = 2 * L + 2 * max_qp + (jmid > 0 ? 2 * jmid : 1);
  double2* Wt = (double2*)smem_d;                        // [2L]: e^{i pi n / L}
  double2* Gt = Wt + 2 * L;                              // [4L + 1]: G(n), n = -2L .. 2L
  const size_t per_warp = (size_t)mmax * (mmax - 1) / 2 * sizeof(double2) + 2 * (size_t)mmax * sizeof(double2) +
                          (size_t)mmax * sizeof(DirOp);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wbase = (unsigned char*)(Gt + 4 * L + 1) + (size_t)warp * per_warp;
  double2* T = (double2*)wbase;
  double2* rowR = T + (size_t)mmax * (mmax - 1) / 2;
  double2* tau = rowR + mmax;
  DirOp* ops = (DirOp*)(tau + mmax);
  for (int n = threadIdx.x; n < 2 * L; n += blockDim.x) {
    double sn, cs;
    sincospi((double)n / L, &sn, &cs);
    Wt[n] = make_double2(cs, sn);
  }
  __syncthreads();
  for (int n = threadIdx.x; n <= 4 * L; n += blockDim.x) {
    const int ph = n - 2 * L;
    double2 g = make_double2(0.0, 0.0);
    for (int j = 1; j <= L; ++j) {
      const double2 w = Wt[wrap2L(ph * j, L)];
      g.x += w.x;
      g.y += w.y;
    }
    Gt[n] = make_double2(g.x / L, g.y / L);
  }
  __syncthreads();
  const double rn = rsqrt((double)L);
  for (int64_t q = (int64_t)blockIdx.x * wpc + warp; q < n_pairs; q += (int64_t)gridDim.x * wpc) {
    const int32_t pa = pairs[2 * q], pb = pairs[2 * q + 1];
    if (pa < 0 || pa >= n_a || pb < 0 || pb >= n_b) {        // warp-uniform
      if (lane == 0) {
        atomicOr(status, kStBadIndex);
        out[2 * q] = out[2 * q + 1] = __longlong_as_double(0x7ff8000000000000ll);
      }
      continue;
    }
    // the operator string (lane 0), each operator as (a, b, ph, loc)
    int m = 0;
    if (lane == 0) {
      const int16_t* sa = (pa_par ? modes_r : modes_ns) + (a_off + pa) * max_qp;
      const int16_t* sb = (pb_par ? modes_r : modes_ns) + (b_off + pb) * max_qp;
      const int oa = pa_par * L, ob = pb_par * L;     // mode tables: NS modes, then R modes
      int ma = 0, mb = 0;
      while (ma < max_qp && sa[ma] >= 0) ++ma;
      while (mb < max_qp && sb[mb] >= 0) ++mb;
      int c = 0;
      auto mode_op = [&](bool dag, int n, double th) {
        double s2, c2;
        sincos(0.5 * th, &s2, &c2);
        DirOp o;
        o.loc = 0;
        if (dag) { o.ph = n; o.a = make_double2(s2, 0.0); o.b = make_double2(0.0, c2); }      // s c_k^dag + i c c_{-k}
        else { o.ph = -n; o.a = make_double2(0.0, -c2); o.b = make_double2(s2, 0.0); }        // s c_k - i c c_{-k}^dag
        ops[c++] = o;
      };
      auto plain_op = [&](bool dag, int n) {           // c_k or c_k^dag at k = pi n / L
        DirOp o;
        o.loc = 0;
        o.ph = dag ? n : -n;
        o.a = make_double2(dag ? 1.0 : 0.0, 0.0);
        o.b = make_double2(dag ? 0.0 : 1.0, 0.0);
        ops[c++] = o;
      };
      auto site_op = [&](int l, double bsign) {        // c_l^dag + bsign c_l
        DirOp o;
        o.loc = l;
        o.ph = 0;
        o.a = make_double2(1.0, 0.0);
        o.b = make_double2(bsign, 0.0);
        ops[c++] = o;
      };
      for (int i = 0; i < L; ++i) {                  // bra vacuum: d_k^dag, ascending (k != pi)
        const int n = nlab[oa + i];
        if (n != L) mode_op(true, n, theta[oa + i]);
      }
      for (int t = ma - 1; t >= 0; --t) {            // bra excitations: d_p, descending ((c_pi^dag)^dag)
        const int i = sa[t], n = nlab[oa + i];
        if (n == L) plain_op(false, L);
        else mode_op(false, n, theta[oa + i]);
      }
      if (jmid < 0) {
        site_op(1, 1.0);                             // sigma^x_1 = c_1 + c_1^dag
      } else {                                       // sigma^x_1 sigma^x_{j+1} = B_1 A_2 B_2 ... B_j A_{j+1}
        for (int l = 1; l <= jmid; ++l) {
          site_op(l, -1.0);
          site_op(l + 1, 1.0);
        }
      }
      for (int t = 0; t < mb; ++t) {                 // ket excitations: d_q^dag (c_pi^dag), ascending
        const int i = sb[t], n = nlab[ob + i];
        if (n == L) plain_op(true, L);
        else mode_op(true, n, theta[ob + i]);
      }
      for (int i = L - 1; i >= 0; --i) {             // ket vacuum: d_k (k != pi), descending
        const int n = nlab[ob + i];
        if (n != L) mode_op(false, n, theta[ob + i]);
      }
      m = c;
    }
    m = __shfl_sync(0xffffffffu, m, 0);
    __syncwarp();
    // A_uv = b_u a_v sum_j phi_u(j) phi_v(j), u < v (Eq. S2), the site sum from the tables
    for (int u = 0; u < m; ++u) {
      const DirOp ou = ops[u];
      for (int v = u + 1 + lane; v < m; v += 32) {
        const DirOp ov = ops[v];
        double2 sj;
        if (ou.loc == 0 && ov.loc == 0) sj = Gt[ou.ph + ov.ph + 2 * L];
        else if (ou.loc == 0) { const double2 w = Wt[wrap2L(ou.ph * ov.loc, L)]; sj = make_double2(w.x * rn, w.y * rn); }
        else if (ov.loc == 0) { const double2 w = Wt[wrap2L(ov.ph * ou.loc, L)]; sj = make_double2(w.x * rn, w.y * rn); }
        else sj = make_double2(ou.loc == ov.loc ? 1.0 : 0.0, 0.0);
        T[pk(u, v, m)] = cmul(cmul(ou.b, ov.a), sj);
      }
    }
    __syncwarp();
    const double2 pf = pf_packed_warp(T, m, rowR, tau, lane);
    if (lane == 0) {
      const double re = vac_norm * pf.x, im = vac_norm * pf.y;
      if (!(isfinite(re) && isfinite(im))) atomicOr(status, kStNan);
      out[2 * q] = re;
      out[2 * q + 1] = im;
    }
    __syncwarp();
  }
}

// <phi_a| B_1 A_2 ... B_j A_{j+1} |phi_b> for pairs of states of one parity from the
// contraction table S of z_table (nE = 2L + 2J operators): the Pfaffian of S over the element's
// operators, m = M_a + 2j + M_b, times c0z = n_P^2 Pf(A_FF).
__global__ void __launch_bounds__(kDirThreads)
z_reduced_kernel(const int32_t* __restrict__ pairs, int64_t n_pairs, int j, int J, int64_t off, int64_t n_states, int L,
                 const double2* __restrict__ S, const double2* __restrict__ c0z, const int16_t* __restrict__ modes,
                 int max_qp, double* __restrict__ out, unsigned* __restrict__ status) {
  extern __shared__ double smem_d[];
  __shared__ int sel[2 * kMaxQp + 2 * kMaxL];
  __shared__ int nsel;
  const int nE = 2 * L + 2 * J;
  const int mmax = 2 * max_qp + 2 * j;
  double2* T = (double2*)smem_d;                 // packed strict upper triangle, m (m - 1) / 2
  double2* rowR = T + (size_t)mmax * (mmax - 1) / 2;
  double2* tau = rowR + mmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = kDirThreads / 32;
  for (int64_t q = blockIdx.x; q < n_pairs; q += gridDim.x) {
    const int32_t pa = pairs[2 * q], pb = pairs[2 * q + 1];
    if (pa < 0 || pa >= n_states || pb < 0 || pb >= n_states) {   // block-uniform
      if (threadIdx.x == 0) {
        atomicOr(status, kStBadIndex);
        out[2 * q] = out[2 * q + 1] = __longlong_as_double(0x7ff8000000000000ll);
      }
      continue;
    }
    if (threadIdx.x == 0) {
      const int16_t* sa = modes + (off + pa) * max_qp;
      const int16_t* sb = modes + (off + pb) * max_qp;
      int ma = 0, mb = 0;
      while (ma < max_qp && sa[ma] >= 0) ++ma;
      while (mb < max_qp && sb[mb] >= 0) ++mb;
      int c = 0;
      for (int t = ma - 1; t >= 0; --t) sel[c++] = L - 1 - sa[t];   // bra excitations, descending
      for (int x = 0; x < 2 * j; ++x) sel[c++] = L + x;            // B_1 A_2 ... B_j A_{j+1}
      for (int t = 0; t < mb; ++t) sel[c++] = L + 2 * J + sb[t];    // ket excitations, ascending
      nsel = c;
    }
    __syncthreads();
    const int m = nsel;
    for (int u = warp; u < m; u += nwarp) {          // a warp per row, lanes along it
      const double2* srow = S + (size_t)sel[u] * nE;
      for (int v = u + 1 + lane; v < m; v += 32) T[pk(u, v, m)] = srow[sel[v]];
    }
    __syncthreads();
    const double2 pf = pf_packed(T, m, rowR, tau);
    if (threadIdx.x == 0) {
      const double2 z = cmul(*c0z, pf);
      if (!(isfinite(z.x) && isfinite(z.y))) atomicOr(status, kStNan);
      out[2 * q] = z.x;
      out[2 * q + 1] = z.y;
    }
    __syncthreads();
  }
}

}  // namespace

size_t z_reduced_smem(int max_qp, int j) {
  const size_t m = (size_t)(2 * max_qp + 2 * j);
  return sizeof(double2) * (m * (m > 0 ? m - 1 : 0) / 2 + 2 * m + 2);
}

// Z elements of explicit pairs of parity `parity` of sector s, 0 <= j <= J, from the table of
// z_table(b, parity, J, S, c0z).  out: complex, interleaved.
tgba_status z_reduced_elements(Basis& b, int s, int parity, int j, int J, const double* S, const double* c0z,
                               const int32_t* pairs, int64_t n, double* out, cudaStream_t st) {
  if (n == 0) return TGBA_OK;
  const Sector& sec = b.sectors[s];
  const size_t smem = z_reduced_smem(b.max_qp, j);
  TGBA_CUDA(cudaFuncSetAttribute(z_reduced_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  const int64_t grid = std::min<int64_t>(n, (int64_t)sms * 16);
  z_reduced_kernel<<<(unsigned)grid, kDirThreads, smem, st>>>(
      pairs, n, j, J, parity ? sec.r_off : sec.ns_off, parity ? sec.n_r : sec.n_ns, b.L, (const double2*)S,
      (const double2*)c0z, parity ? b.d_modes_r : b.d_modes_ns, b.max_qp, out, b.d_status);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

// shared memory of one warp's element (string, packed triangle, scratch) and of the CTA tables
size_t x_direct_warp_smem(int L, int max_qp, int jmid) {
  const size_t m = (size_t)(2 * L + 2 * max_qp + (jmid > 0 ? 2 * jmid : 1));
  return sizeof(double2) * (m * (m - 1) / 2 + 2 * m) + sizeof(DirOp) * m;
}
size_t x_direct_smem(int L, int max_qp, int jmid) {       // one warp per CTA: the least that must fit
  return sizeof(double2) * (size_t)(6 * L + 1) + x_direct_warp_smem(L, max_qp, jmid);
}

// Elements <phi_a|O|phi_b> for explicit (a, b) pairs of sector s: O = sigma^x_1 between NS bra
// and R ket (jmid < 0), or sigma^x_1 sigma^x_{jmid+1} between two states of parity `parity`.
tgba_status direct_elements(Basis& b, int s, int parity, int jmid, const int32_t* pairs, int64_t n, double* out,
                            cudaStream_t st) {
  if (n == 0) return TGBA_OK;
  const Sector& sec = b.sectors[s];
  // warps per CTA: as many elements as fit in about half of an SM's shared memory (two CTAs
  // per SM), at most 8
  int limit = 0, sms = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.device));
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device));
  const size_t tables = sizeof(double2) * (size_t)(6 * b.L + 1), per_warp = x_direct_warp_smem(b.L, b.max_qp, jmid);
  if (tables + per_warp > (size_t)limit) return fail(TGBA_EINVAL, "direct string does not fit in shared memory");
  const int wpc = (int)std::max<size_t>(1, std::min<size_t>(8, ((size_t)limit / 2 - tables) / per_warp));
  const size_t smem = tables + (size_t)wpc * per_warp;
  TGBA_CUDA(cudaFuncSetAttribute(x_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TGBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, x_direct_kernel, 32 * wpc, smem));
  const int64_t grid = std::min<int64_t>((n + wpc - 1) / wpc, (int64_t)sms * std::max(1, per_sm));
  const int pa_par = jmid < 0 ? 0 : parity, pb_par = jmid < 0 ? 1 : parity;
  const int64_t a_off = pa_par ? sec.r_off : sec.ns_off, b_off = pb_par ? sec.r_off : sec.ns_off;
  const int64_t n_a = pa_par ? sec.n_r : sec.n_ns, n_b = pb_par ? sec.n_r : sec.n_ns;
  const double norm = jmid < 0 ? b.vac_norm : (parity ? b.norm_r * b.norm_r : b.norm_ns * b.norm_ns);
  x_direct_kernel<<<(unsigned)grid, 32 * wpc, smem, st>>>(pairs, n, pa_par, pb_par, jmid, a_off, b_off, n_a, n_b, b.L,
                                                          b.d_theta, b.d_nlab, b.d_modes_ns, b.d_modes_r, b.max_qp,
                                                          norm, wpc, out, b.d_status);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

tgba_status x_direct(Basis& b, int s, const int32_t* pairs, int64_t n, double* out, cudaStream_t st) {
  return direct_elements(b, s, 0, -1, pairs, n, out, st);
}

}  // namespace tgba
