/*
 * TGBA oracle, C part.  TEST INFRASTRUCTURE ONLY: it is imported by the tests, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline leg, never by the product path.
 *
 * What it computes, plainly and slowly, in complex double precision:
 *
 *  1. Wick's theorem as a Pfaffian (Appendix A, Eq. S1-S2).  Each operator is a linear
 *     combination O_m = sum_j (U_jm c_j^dag + V_jm c_j) over the N Jordan-Wigner fermions.
 *     The vacuum expectation <0|O_1 ... O_2n|0>_c is Pf(A), where A is skew-symmetric and
 *     its strict upper triangle is that of V^T U.
 *
 *  2. The Pfaffian itself by Parlett-Reid reduction with partial pivoting (the O((2n)^3)
 *     class of algorithm the paper cites, Wimmer 2012): eliminate two rows/columns per
 *     step, choosing as pivot the largest entry of the current column.
 *
 * The operator kinds are the ones the Ising example needs (Eq. 6-7 and Appendix A):
 *   c_k      = N^{-1/2} sum_j e^{-ikj} c_j
 *   c_k^dag  = N^{-1/2} sum_j e^{+ikj} c_j^dag
 *   d_k      = sin(theta/2) c_k - i cos(theta/2) c_{-k}^dag
 *   d_k^dag  = sin(theta/2) c_k^dag + i cos(theta/2) c_{-k}
 *   sigma    = c_1 + c_1^dag   (sigma^x on site 1, no Jordan-Wigner string)
 * Sites run j = 1..N.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

enum { OP_C = 0, OP_CDAG = 1, OP_D = 2, OP_DDAG = 3, OP_SIGMA1 = 4, OP_MAJ_A = 5, OP_MAJ_B = 6 };
/* OP_MAJ_A / OP_MAJ_B: the Majorana operators c_l^dag + c_l and c_l^dag - c_l of site l = (int)k */

/* Pfaffian of the dense skew-symmetric n x n matrix A (row-major; destroyed). */
cplx oracle_pfaffian(cplx* A, int n) {
  if (n == 0) return 1.0;
  if (n % 2) return 0.0;
  cplx pf = 1.0;
  for (int k = 0; k < n - 1; k += 2) {
    /* pivot: largest |A[i][k]|, i > k */
    int piv = k + 1;
    double best = cabs(A[(size_t)(k + 1) * n + k]);
    for (int i = k + 2; i < n; ++i) {
      double v = cabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; piv = i; }
    }
    if (piv != k + 1) {
      /* symmetric swap of rows and columns k+1 <-> piv: one transposition, sign flips */
      for (int j = 0; j < n; ++j) {
        cplx t = A[(size_t)(k + 1) * n + j];
        A[(size_t)(k + 1) * n + j] = A[(size_t)piv * n + j];
        A[(size_t)piv * n + j] = t;
      }
      for (int i = 0; i < n; ++i) {
        cplx t = A[(size_t)i * n + (k + 1)];
        A[(size_t)i * n + (k + 1)] = A[(size_t)i * n + piv];
        A[(size_t)i * n + piv] = t;
      }
      pf = -pf;
    }
    cplx a = A[(size_t)k * n + (k + 1)];
    if (a == 0.0) return 0.0;
    pf *= a;
    /* Schur complement of the 2x2 pivot block [[0,a],[-a,0]] on the trailing block:
       A_ij += (A[k+1][i] A[k][j] - A[k][i] A[k+1][j]) / a,  i, j >= k+2 */
    for (int i = k + 2; i < n; ++i) {
      cplx r1i = A[(size_t)(k + 1) * n + i], r0i = A[(size_t)k * n + i];
      for (int j = k + 2; j < n; ++j) {
        cplx r0j = A[(size_t)k * n + j], r1j = A[(size_t)(k + 1) * n + j];
        A[(size_t)i * n + j] += (r1i * r0j - r0i * r1j) / a;
      }
    }
  }
  return pf;
}

/* Coefficients (U_j, V_j), j = 1..N stored at index j-1, of one operator. */
static void op_coeffs(int N, int kind, double k, double theta, cplx* U, cplx* V) {
  const double s = sin(0.5 * theta), c = cos(0.5 * theta), rn = 1.0 / sqrt((double)N);
  for (int j = 1; j <= N; ++j) {
    cplx ep = cexp(I * k * j) * rn, em = cexp(-I * k * j) * rn;
    cplx u = 0.0, v = 0.0;
    switch (kind) {
      case OP_C:      v = em; break;
      case OP_CDAG:   u = ep; break;
      case OP_D:      v = s * em; u = -I * c * em; break;    /* c_{-k}^dag carries e^{-ikj} */
      case OP_DDAG:   u = s * ep; v = I * c * ep; break;     /* c_{-k} carries e^{+ikj} */
      case OP_SIGMA1: u = (j == 1) ? 1.0 : 0.0; v = u; break;
      case OP_MAJ_A: u = (j == (int)k) ? 1.0 : 0.0; v = u; break;
      case OP_MAJ_B: u = (j == (int)k) ? 1.0 : 0.0; v = -u; break;
    }
    U[j - 1] = u; V[j - 1] = v;
  }
}

/* <0|O_1...O_m|0>_c for one operator string (Eq. S1-S2). */
static cplx wick_string(int N, int m, const int* kinds, const double* ks, const double* th,
                        cplx* U, cplx* V, cplx* A) {
  if (m % 2) return 0.0;
  for (int a = 0; a < m; ++a) op_coeffs(N, kinds[a], ks[a], th[a], U + (size_t)a * N, V + (size_t)a * N);
  for (int a = 0; a < m; ++a) {
    A[(size_t)a * m + a] = 0.0;
    for (int b = a + 1; b < m; ++b) {
      cplx acc = 0.0;                       /* (V^T U)_{ab} = sum_j V_ja U_jb */
      for (int j = 0; j < N; ++j) acc += V[(size_t)a * N + j] * U[(size_t)b * N + j];
      A[(size_t)a * m + b] = acc;
      A[(size_t)b * m + a] = -acc;
    }
  }
  return oracle_pfaffian(A, m);
}

/* Batch of operator strings.  String s occupies entries offsets[s] .. offsets[s+1]-1 of
   kinds/ks/thetas.  out[s] = <0|O...O|0>_c.  Returns the number of threads used. */
int oracle_wick_batch(int N, int n_strings, const long long* offsets, const int* kinds,
                      const double* ks, const double* thetas, double* out_ri, int n_threads) {
  int used = 1;
#ifdef _OPENMP
  omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
  }
#endif
  int mmax = 0;
  for (int s = 0; s < n_strings; ++s) {
    int m = (int)(offsets[s + 1] - offsets[s]);
    if (m > mmax) mmax = m;
  }
#pragma omp parallel
  {
    cplx* U = (cplx*)malloc(sizeof(cplx) * (size_t)(mmax > 0 ? mmax : 1) * N);
    cplx* V = (cplx*)malloc(sizeof(cplx) * (size_t)(mmax > 0 ? mmax : 1) * N);
    cplx* A = (cplx*)malloc(sizeof(cplx) * (size_t)(mmax > 0 ? mmax : 1) * (mmax > 0 ? mmax : 1));
#pragma omp for schedule(dynamic, 4)
    for (int s = 0; s < n_strings; ++s) {
      long long o = offsets[s];
      int m = (int)(offsets[s + 1] - o);
      cplx r = wick_string(N, m, kinds + o, ks + o, thetas + o, U, V, A);
      out_ri[2 * (size_t)s] = creal(r);
      out_ri[2 * (size_t)s + 1] = cimag(r);
    }
    free(U); free(V); free(A);
  }
  return used;
}

/* Pfaffians of a batch of dense skew matrices (row-major, each n x n, overwritten). */
void oracle_pfaffian_batch(int n, int count, double* mats_ri, double* out_ri) {
  for (int c = 0; c < count; ++c) {
    cplx r = oracle_pfaffian((cplx*)(mats_ri + 2 * (size_t)c * n * n), n);
    out_ri[2 * (size_t)c] = creal(r);
    out_ri[2 * (size_t)c + 1] = cimag(r);
  }
}

/* ------------------------------------------------------------------ reduced form
 * The same elements through the Schur complement identity for Pfaffians: for a skew matrix
 * [[A_FF, A_FE], [-A_FE^T, A_EE]] with A_FF invertible,
 *   Pf = Pf(A_FF) Pf(A_EE + A_FE^T A_FF^{-1} A_FE).
 * Every element's operator string keeps the same operators F (both vacua and sigma) and adds
 * the excitation operators of its two states, so with S = A_EE + A_FE^T A_FF^{-1} A_FE over ALL
 * excitation operators E, an element is Pf(A_FF) Pf(S[sel, sel]) (moving F to the front of the
 * string costs a sign (-1)^{M + (N-1)(M+M')} = +1 for even M, M').  A second, independent CPU
 * route to the same numbers (it shares only op_coeffs and oracle_pfaffian with the direct one),
 * used as the faster CPU baseline. */

/* A over one string of m operators (strict upper triangle of V^T U, made skew), row-major. */
static void contraction_matrix(int N, int m, const int* kinds, const double* ks, const double* th, cplx* A) {
  cplx* U = (cplx*)malloc(sizeof(cplx) * (size_t)m * N);
  cplx* V = (cplx*)malloc(sizeof(cplx) * (size_t)m * N);
  for (int a = 0; a < m; ++a) op_coeffs(N, kinds[a], ks[a], th[a], U + (size_t)a * N, V + (size_t)a * N);
  for (int a = 0; a < m; ++a) {
    A[(size_t)a * m + a] = 0.0;
    for (int b = a + 1; b < m; ++b) {
      cplx acc = 0.0;
      for (int j = 0; j < N; ++j) acc += V[(size_t)a * N + j] * U[(size_t)b * N + j];
      A[(size_t)a * m + b] = acc;
      A[(size_t)b * m + a] = -acc;
    }
  }
  free(U);
  free(V);
}

/* Table of the reduced form.  The string has m operators; is_f[a] = 1 marks the F operators.
   Writes S (nE x nE, row-major, E operators in string order) and Pf(A_FF) (re, im).  Returns 0,
   or 1 if A_FF is singular. */
int oracle_reduced_table(int N, int m, const int* kinds, const double* ks, const double* th, const int* is_f,
                         double* S_ri, double* pf_ri) {
  cplx* A = (cplx*)malloc(sizeof(cplx) * (size_t)m * m);
  contraction_matrix(N, m, kinds, ks, th, A);
  int nF = 0;
  for (int a = 0; a < m; ++a) nF += is_f[a] != 0;
  const int nE = m - nF;
  int* fi = (int*)malloc(sizeof(int) * (nF > 0 ? nF : 1));
  int* ei = (int*)malloc(sizeof(int) * (nE > 0 ? nE : 1));
  for (int a = 0, f = 0, e = 0; a < m; ++a) {
    if (is_f[a]) fi[f++] = a;
    else ei[e++] = a;
  }
  /* Z = A_FF^{-1} A_FE by Gaussian elimination with partial pivoting on [A_FF | A_FE] */
  cplx* M = (cplx*)malloc(sizeof(cplx) * (size_t)nF * (nF + nE));
  const int w = nF + nE;
  for (int r = 0; r < nF; ++r) {
    for (int c = 0; c < nF; ++c) M[(size_t)r * w + c] = A[(size_t)fi[r] * m + fi[c]];
    for (int c = 0; c < nE; ++c) M[(size_t)r * w + nF + c] = A[(size_t)fi[r] * m + ei[c]];
  }
  int singular = 0;
  for (int k = 0; k < nF && !singular; ++k) {
    int piv = k;
    for (int r = k + 1; r < nF; ++r)
      if (cabs(M[(size_t)r * w + k]) > cabs(M[(size_t)piv * w + k])) piv = r;
    if (M[(size_t)piv * w + k] == 0.0) { singular = 1; break; }
    if (piv != k)
      for (int c = 0; c < w; ++c) {
        cplx t = M[(size_t)k * w + c];
        M[(size_t)k * w + c] = M[(size_t)piv * w + c];
        M[(size_t)piv * w + c] = t;
      }
    for (int r = 0; r < nF; ++r) {
      if (r == k) continue;
      const cplx f = M[(size_t)r * w + k] / M[(size_t)k * w + k];
      if (f == 0.0) continue;
      for (int c = k; c < w; ++c) M[(size_t)r * w + c] -= f * M[(size_t)k * w + c];
    }
  }
  if (!singular) {
    /* S = A_EE + A_FE^T Z, Z[r][c] = M[r][nF + c] / M[r][r] */
    for (int i = 0; i < nE; ++i)
      for (int j = 0; j < nE; ++j) {
        cplx acc = A[(size_t)ei[i] * m + ei[j]];
        for (int r = 0; r < nF; ++r)
          acc += A[(size_t)fi[r] * m + ei[i]] * (M[(size_t)r * w + nF + j] / M[(size_t)r * w + r]);
        S_ri[2 * ((size_t)i * nE + j)] = creal(acc);
        S_ri[2 * ((size_t)i * nE + j) + 1] = cimag(acc);
      }
    cplx* F = (cplx*)malloc(sizeof(cplx) * (size_t)(nF > 0 ? nF : 1) * (nF > 0 ? nF : 1));
    for (int r = 0; r < nF; ++r)
      for (int c = 0; c < nF; ++c) F[(size_t)r * nF + c] = A[(size_t)fi[r] * m + fi[c]];
    cplx p = oracle_pfaffian(F, nF);
    pf_ri[0] = creal(p);
    pf_ri[1] = cimag(p);
    free(F);
  }
  free(M); free(fi); free(ei); free(A);
  return singular;
}

/* out[p] = scale Pf(A_FF) Pf(S[sel_p, sel_p]) for each pair p; sel_p = idx[off[p] .. off[p+1]-1]
   (positions in E, ascending).  Returns the number of threads used. */
int oracle_reduced_batch(int nE, const double* S_ri, const double* pf_ri, double scale, int n_pairs,
                         const long long* off, const int* idx, double* out_ri, int n_threads) {
  int used = 1;
#ifdef _OPENMP
  omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
  }
#endif
  const cplx* S = (const cplx*)S_ri;
  const cplx pf = (pf_ri[0] + I * pf_ri[1]) * scale;
  int nmax = 0;
  for (int p = 0; p < n_pairs; ++p) {
    int n = (int)(off[p + 1] - off[p]);
    if (n > nmax) nmax = n;
  }
#pragma omp parallel
  {
    cplx* B = (cplx*)malloc(sizeof(cplx) * (size_t)(nmax > 0 ? nmax * nmax : 1));
#pragma omp for schedule(dynamic, 256)
    for (int p = 0; p < n_pairs; ++p) {
      const int* sel = idx + off[p];
      const int n = (int)(off[p + 1] - off[p]);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) B[(size_t)i * n + j] = S[(size_t)sel[i] * nE + sel[j]];
      const cplx r = pf * oracle_pfaffian(B, n);
      out_ri[2 * (size_t)p] = creal(r);
      out_ri[2 * (size_t)p + 1] = cimag(r);
    }
    free(B);
  }
  return used;
}
