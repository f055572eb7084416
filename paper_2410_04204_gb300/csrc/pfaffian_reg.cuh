// Register-resident Pfaffian of a fixed small size N (N <= 14): the strict upper triangle of the
// N x N skew matrix lives in registers, every index is a compile-time constant, and the row/
// column exchange of partial pivoting is a chain of predicated selects over the candidate rows.
// FP64 instructions: per elimination step with trailing size m, m(m-1) FMAs (the rank-2 update),
// m multiplies (the Gauss vector), one reciprocal and one multiply (the running Pfaffian).
#pragma once

#include <cstdint>

namespace tgba {

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// sign flip and zero / finiteness tests on the bit pattern: integer ops, off the FP64 pipe
__device__ __forceinline__ double neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ bool is_zero(double x) { return abs_bits(x) == 0ull; }
__device__ __forceinline__ bool is_finite_bits(double x) { return abs_bits(x) < 0x7ff0000000000000ull; }

__device__ __forceinline__ void cswap(bool s, double& a, double& b) {
  const double x = a, y = b;
  a = s ? y : x;
  b = s ? x : y;
}

__device__ __forceinline__ void cswap_neg(bool s, double& a, double& b) {
  const double x = a, y = b;
  a = s ? neg(y) : x;
  b = s ? neg(x) : y;
}

// If s: exchange rows/columns R and C (R < C) of the trailing matrix (rows >= K, R = K + 1).
template <int N, int K, int C>
__device__ __forceinline__ void exchange(bool s, double (&W)[N][N]) {
  constexpr int R = K + 1;
  cswap(s, W[K][R], W[K][C]);
#pragma unroll
  for (int x = R + 1; x < C; ++x) cswap_neg(s, W[R][x], W[x][C]);
  W[R][C] = s ? neg(W[R][C]) : W[R][C];
#pragma unroll
  for (int x = C + 1; x < N; ++x) cswap(s, W[R][x], W[C][x]);
}

template <int N, int K, int C>
struct ExchangeAll {
  static __device__ __forceinline__ void run(int p, double (&W)[N][N]) {
    exchange<N, K, C>(p == C, W);
    ExchangeAll<N, K, C + 1>::run(p, W);
  }
};
template <int N, int K>
struct ExchangeAll<N, K, N> {
  static __device__ __forceinline__ void run(int, double (&)[N][N]) {}
};

template <int N, int K>
struct Eliminate {
  static __device__ __forceinline__ void run(double (&W)[N][N], double& pf) {
    constexpr int R = K + 1;
    // pivot: largest |W[K][x]|, x > K (integer comparison of the magnitudes' bit patterns)
    int p = R;
    unsigned long long best = abs_bits(W[K][R]);
#pragma unroll
    for (int x = R + 1; x < N; ++x) {
      const unsigned long long v = abs_bits(W[K][x]);
      if (v > best) { best = v; p = x; }
    }
    ExchangeAll<N, K, R + 1>::run(p, W);
    const double a = W[K][R];
    pf = (p != R) ? neg(pf) : pf;
    pf *= a;
    if (K + 2 < N) {
      const double ia = is_zero(a) ? 0.0 : __drcp_rn(a);   // a == 0: whole column zero, pf is already 0
#pragma unroll
      for (int j = K + 2; j < N; ++j) W[K][j] *= ia;       // Gauss vector tau_j
#pragma unroll
      for (int i = K + 2; i < N; ++i) {
#pragma unroll
        for (int j = i + 1; j < N; ++j) {
          // W_ij += W(R, i) tau_j - tau_i W(R, j)
          W[i][j] = fma(W[R][i], W[K][j], fma(-W[K][i], W[R][j], W[i][j]));
        }
      }
      Eliminate<N, K + 2>::run(W, pf);
    }
  }
};
template <int N>
struct Eliminate<N, N> {
  static __device__ __forceinline__ void run(double (&)[N][N], double&) {}
};

template <int N>
__device__ __forceinline__ double pfaffian_regs(double (&W)[N][N]) {
  double pf = 1.0;
  Eliminate<N, 0>::run(W, pf);
  return pf;
}

}  // namespace tgba
