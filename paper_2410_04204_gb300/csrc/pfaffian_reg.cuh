// Register-resident Pfaffian of a fixed small size N (N <= 14): the strict upper triangle of the
// N x N skew matrix lives in registers, every index is a compile-time constant, and the row/
// column exchange of partial pivoting is a chain of predicated selects over the candidate rows.
// FP64 instructions: per elimination step with trailing size m, m(m-1) FMAs (the rank-2 update),
// m multiplies (the Gauss vector), one reciprocal and one multiply (the running Pfaffian).
#pragma once

#include <cstdint>

namespace tgba {

// The magnitude's bit pattern, as an integer AND in inline PTX: written in C++ the compiler
// recognises the sign-bit mask as fabs and issues it on the FP64 pipe (measured: one DADD per
// pivot candidate).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  unsigned long long r;
  asm("and.b64 %0, %1, 0x7fffffffffffffff;" : "=l"(r) : "l"((unsigned long long)__double_as_longlong(x)));
  return r;
}

// Every data movement of the pivot exchange is an integer select of the 64-bit pattern, written
// in inline PTX (selp.b64) so that the result is born as one 64-bit register pair: a select
// written as a double select, or as two 32-bit selects reassembled into a double, was measured
// to cost one FP64-pipe instruction (a DADD) per selected operand of a later FP64 operation.
__device__ __forceinline__ double sel(bool s, double y, double x) {        // s ? y : x
  unsigned long long r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\tselp.b64 %0, %1, %2, p;\n\t}"
      : "=l"(r)
      : "l"((unsigned long long)__double_as_longlong(y)), "l"((unsigned long long)__double_as_longlong(x)),
        "r"((int)s));
  return __longlong_as_double((long long)r);
}
// The sign-bit XOR is written in inline PTX: as plain C++ the compiler recognises it as a
// (conditional) floating-point negation and issues it on the FP64 pipe.
__device__ __forceinline__ double flip_if(bool s, double x) {               // s ? -x : x
  const unsigned m = s ? 0x80000000u : 0u;
  double r;
  asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\txor.b32 hi, hi, %2;\n\tmov.b64 %0, {lo, hi};\n\t}"
      : "=d"(r) : "d"(x), "r"(m));
  return r;
}
__device__ __forceinline__ double neg(double x) { return flip_if(true, x); }
__device__ __forceinline__ bool is_zero(double x) { return abs_bits(x) == 0ull; }
__device__ __forceinline__ bool is_finite_bits(double x) { return abs_bits(x) < 0x7ff0000000000000ull; }

// 1/a for the pivot: a single-precision seed, then two Newton-Raphson steps for f(x) = 1/x - a,
// x <- x + x (1 - a x), each squaring the relative error (2^-22 -> 2^-44 -> below double
// rounding).  The seed is built from the double's bit fields with integer operations (sign,
// exponent rebased from 1023 to 127, top 23 mantissa bits) and its reciprocal taken in FP32, so
// the FP64 pipe sees only the four FMAs.  |a| outside [2^-100, 2^100] (never a usable pivot
// here, but possible in principle) takes the library reciprocal instead.
__device__ __forceinline__ double recip_nr(double a) {
  const int hi = __double2hiint(a), lo = __double2loint(a);
  const int e = (hi >> 20) & 0x7ff;
  if (e < 1023 - 100 || e > 1023 + 100) return __drcp_rn(a);
  const unsigned fbits = ((unsigned)hi & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23) |
                         (((unsigned)hi & 0x000fffffu) << 3) | ((unsigned)lo >> 29);
  const float rf = __frcp_rn(__uint_as_float(fbits));
  // back to double bits: sign, exponent rebased from 127 to 1023, mantissa widened
  const unsigned rb = __float_as_uint(rf);
  const int re = (int)((rb >> 23) & 0xff) - 127 + 1023;
  double x = __hiloint2double((int)((rb & 0x80000000u) | ((unsigned)re << 20) | ((rb & 0x7fffffu) >> 3)),
                              (int)(rb << 29));
  double err = fma(-a, x, 1.0);
  x = fma(x, err, x);
  err = fma(-a, x, 1.0);
  return fma(x, err, x);
}

__device__ __forceinline__ void cswap(bool s, double& a, double& b) {
  const double x = a, y = b;
  a = sel(s, y, x);
  b = sel(s, x, y);
}

__device__ __forceinline__ void cswap_neg(bool s, double& a, double& b) {
  const double x = a, y = b;
  a = sel(s, neg(y), x);
  b = sel(s, neg(x), y);
}

// If s: exchange rows/columns R and C (R < C) of the trailing matrix (rows >= K, R = K + 1).
template <int N, int K, int C>
__device__ __forceinline__ void exchange(bool s, double (&W)[N][N]) {
  constexpr int R = K + 1;
  cswap(s, W[K][R], W[K][C]);
#pragma unroll
  for (int x = R + 1; x < C; ++x) cswap_neg(s, W[R][x], W[x][C]);
  W[R][C] = flip_if(s, W[R][C]);
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
  // pf: product of the pivots; odd: parity of the exchanges (the sign is applied once at the end)
  static __device__ __forceinline__ void run(double (&W)[N][N], double& pf, unsigned& odd) {
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
    odd ^= (p != R) ? 1u : 0u;
    pf *= a;
    if (K + 2 < N) {
      const double ia = sel(is_zero(a), 0.0, recip_nr(a));   // a == 0: whole column zero, pf is already 0
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
      Eliminate<N, K + 2>::run(W, pf, odd);
    }
  }
};
template <int N>
struct Eliminate<N, N> {
  static __device__ __forceinline__ void run(double (&)[N][N], double&, unsigned&) {}
};

template <int N>
__device__ __forceinline__ double pfaffian_regs(double (&W)[N][N]) {
  double pf = 1.0;
  unsigned odd = 0;
  Eliminate<N, 0>::run(W, pf, odd);
  return flip_if(odd != 0, pf);
}

}  // namespace tgba
