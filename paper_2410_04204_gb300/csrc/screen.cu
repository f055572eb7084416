// Learned pair screener (rows a5 and a5' of the hot path; not in the paper, asked for by the
// benchmark configuration): a 3-layer MLP, width H, predicting log10|X_ab| from the two
// quasiparticle momentum sets, trained on exact elements of the Pfaffian path by the kernels of
// this file, and used to skip the Pfaffians of pairs predicted negligible.
//
// Features (D = 2Q + 4, Q = 8): k/pi of the NS state's modes (ascending, zero padded), k/pi of
// the R state's modes, M_a/Q, M_b/Q, 24/L, 1.  Target: log10|X| + (M_a + M_b)/2 log10(L/24),
// clipped at -30 (the 1/sqrt(L) normalisation of each quasiparticle taken out).
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3, MSE loss, Adam.
// Parameters (FP32) are stored flat as W1 [H][D], b1, W2 [H][H], b2, w3, b3.
//
// Training runs in FP32 on the CUDA cores (tiled SGEMM below).  Inference factors layer 1 into
// per-state partials, h1(a, b) = relu(A_a + B_b) with A_a = W1[:, NS part] x_a and
// B_b = W1[:, R part] x_b + b1, and runs layer 2 on the tensor cores (tcgen05 MMAs, BF16
// inputs, FP32 accumulation in tensor memory; screen_tc.cu), fused with the ReLU, the dot with
// w3, the threshold and the compaction of the kept pairs into per-size work lists.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "tgba_internal.h"

namespace tgba {

constexpr int kQ = 8;
constexpr int kD = 2 * kQ + 4;

struct Screen {
  int H = 256;
  int64_t P = 0;
  float* theta = nullptr;   // parameters
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  __nv_bfloat16* W2b = nullptr;   // W2 in BF16 for inference, [H][H] row-major (output, input)
  bool w2b_valid = false;
  double margin = 1.0, val_rmse = 0, train_rmse = 0;
  int64_t adam_step = 0;
  int device = 0;
};

namespace {

// ----------------------------------------------------------------------------- SGEMM (FP32)
// C[M][N] = op(A) op(B) (+ C if accumulate), all row-major.  op(A) is A [M][K] or, if TA,
// A^T with A stored [K][M]; op(B) is B [K][N] or, if TB, B^T with B stored [N][K].
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm(int M, int N, int K, const float* __restrict__ A,
                                             const float* __restrict__ B, float* __restrict__ C) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int r = row0 + mm, k = k0 + kk, c = col0 + mm;
      float a = 0.f, b = 0.f;
      if (r < M && k < K) a = TA ? A[(size_t)k * M + r] : A[(size_t)r * K + k];
      if (c < N && k < K) b = TB ? B[(size_t)c * K + k] : B[(size_t)k * N + c];
      As[kk][mm] = a;
      Bs[kk][mm] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = row0 + ty * 4 + i, c = col0 + tx * 4 + j;
      if (r < M && c < N) C[(size_t)r * N + c] = acc[i][j];
    }
}

template <bool TA, bool TB>
void gemm(cudaStream_t st, int M, int N, int K, const float* A, const float* B, float* C) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  sgemm<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, B, C);
}

// Z += bias (per column), H = relu(Z)
__global__ void bias_relu(int64_t rows, int cols, float* __restrict__ Z, const float* __restrict__ bias,
                          float* __restrict__ Hout) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += (int64_t)gridDim.x * blockDim.x) {
    const float z = Z[i] + bias[i % cols];
    Z[i] = z;
    Hout[i] = fmaxf(z, 0.f);
  }
}

// y = H2 w3 + b3, r = y - t (per row), warp per row
__global__ void out_layer(int64_t rows, int H, const float* __restrict__ H2, const float* __restrict__ w3,
                          const float* __restrict__ b3, const float* __restrict__ t, float* __restrict__ y,
                          float* __restrict__ r) {
  const int lane = threadIdx.x & 31;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
       row += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float acc = 0.f;
    for (int j = lane; j < H; j += 32) acc = fmaf(H2[row * H + j], w3[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const float yy = acc + b3[0];
      y[row] = yy;
      if (t) r[row] = yy - t[row];
    }
  }
}

// dZ2 = (dy w3^T) * (Z2 > 0), dy = 2 r / B
__global__ void back_out(int64_t rows, int H, const float* __restrict__ r, const float* __restrict__ w3,
                         const float* __restrict__ Z2, float scale, float* __restrict__ dZ2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * H; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / H;
    const int j = (int)(i - row * H);
    dZ2[i] = Z2[i] > 0.f ? scale * r[row] * w3[j] : 0.f;
  }
}

__global__ void relu_mask(int64_t n, float* __restrict__ d, const float* __restrict__ Z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(Z[i] > 0.f)) d[i] = 0.f;
}

// column sums of a rows x cols matrix (out[j] = scale * sum_i M[i][j]); one thread per column
__global__ void col_sum(int64_t rows, int cols, const float* __restrict__ Mx, float scale, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float acc = 0.f;
  for (int64_t i = 0; i < rows; ++i) acc += Mx[i * cols + j];
  out[j] = scale * acc;
}

// dw3 = H2^T dy, db3 = sum dy  (dy = scale * r)
__global__ void grad_out(int64_t rows, int H, const float* __restrict__ H2, const float* __restrict__ r, float scale,
                         float* __restrict__ dw3, float* __restrict__ db3) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > H) return;
  float acc = 0.f;
  if (j < H) {
    for (int64_t i = 0; i < rows; ++i) acc = fmaf(H2[i * H + j], r[i], acc);
    dw3[j] = scale * acc;
  } else {
    for (int64_t i = 0; i < rows; ++i) acc += r[i];
    db3[0] = scale * acc;
  }
}

__global__ void sum_squares(int64_t n, const float* __restrict__ r, double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)r[i] * r[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void adam_kernel(int64_t n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// features of explicit pairs of one sector (see the file header)
__global__ void pair_features(int64_t n, const int32_t* __restrict__ pairs, int64_t ns_off, int64_t r_off,
                              const int16_t* __restrict__ modes_ns, const int16_t* __restrict__ modes_r,
                              const uint8_t* __restrict__ M_ns, const uint8_t* __restrict__ M_r, int max_qp,
                              const int* __restrict__ nlab, int L, float* __restrict__ x) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = ns_off + pairs[2 * q], b = r_off + pairs[2 * q + 1];
    float* xr = x + q * kD;
    for (int i = 0; i < kD; ++i) xr[i] = 0.f;
    const int ma = M_ns[a], mb = M_r[b];
    for (int i = 0; i < ma && i < kQ; ++i) xr[i] = (float)nlab[modes_ns[a * max_qp + i]] / L;
    for (int i = 0; i < mb && i < kQ; ++i) xr[kQ + i] = (float)nlab[L + modes_r[b * max_qp + i]] / L;
    xr[2 * kQ] = (float)ma / kQ;
    xr[2 * kQ + 1] = (float)mb / kQ;
    xr[2 * kQ + 2] = 24.f / L;
    xr[2 * kQ + 3] = 1.f;
  }
}

// training targets from exact X (complex, interleaved)
__global__ void pair_targets(int64_t n, const int32_t* __restrict__ pairs, int64_t ns_off, int64_t r_off,
                             const uint8_t* __restrict__ M_ns, const uint8_t* __restrict__ M_r,
                             const double* __restrict__ X, double log_l_ratio, float* __restrict__ t) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double ax = hypot(X[2 * q], X[2 * q + 1]);
    const int nq = M_ns[ns_off + pairs[2 * q]] + M_r[r_off + pairs[2 * q + 1]];
    double y = ax > 0 ? log10(ax) : -30.0;
    y = fmax(y + 0.5 * nq * log_l_ratio, -30.0);
    t[q] = (float)y;
  }
}

__global__ void gather_rows(int64_t n, int D, const int64_t* __restrict__ idx, const float* __restrict__ x,
                            const float* __restrict__ t, float* __restrict__ xb, float* __restrict__ tb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * D; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / D;
    const int c = (int)(i - r * D);
    xb[i] = x[idx[r] * D + c];
    if (c == 0) tb[r] = t[idx[r]];
  }
}

__global__ void to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// ----------------------------------------------------------------------------- inference
// Per-state layer-1 partials.  NS: A_a = W1[:, 0:Q] x_a + W1[:, 2Q] M_a/Q.
// R: B_b = W1[:, Q:2Q] x_b + W1[:, 2Q+1] M_b/Q + W1[:, 2Q+2] 24/L + W1[:, 2Q+3] + b1.
__global__ void state_partials(int64_t n_states, bool ns, const int16_t* __restrict__ modes,
                               const uint8_t* __restrict__ Mq, int max_qp, const int* __restrict__ nlab, int L, int H,
                               const float* __restrict__ W1, const float* __restrict__ b1, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_states * H; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / H;
    const int o = (int)(i - s * H);
    const int M = Mq[s];
    const float* w = W1 + (size_t)o * kD;
    float acc;
    if (ns) {
      acc = w[2 * kQ] * ((float)M / kQ);
      for (int q = 0; q < M && q < kQ; ++q) acc = fmaf(w[q], (float)nlab[modes[s * max_qp + q]] / L, acc);
    } else {
      acc = b1[o] + w[2 * kQ + 1] * ((float)M / kQ) + w[2 * kQ + 2] * (24.f / L) + w[2 * kQ + 3];
      for (int q = 0; q < M && q < kQ; ++q) acc = fmaf(w[kQ + q], (float)nlab[L + modes[s * max_qp + q]] / L, acc);
    }
    out[i] = acc;
  }
}

int blocks(int64_t work, int t = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + t - 1) / t, 152 * 16));
}

// SplitMix64 (Steele, Lea, Flood 2014): the counter-based generator of the training sample.
uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

}  // namespace

// ----------------------------------------------------------------------------- host side
tgba_status screen_create(int H, const float* params, uint64_t seed, Screen** out) {
  Screen* s = new Screen();
  s->H = H;
  s->P = (int64_t)H * kD + H + (int64_t)H * H + H + H + 1;
  cudaGetDevice(&s->device);
  std::vector<float> th(s->P, 0.f);
  if (params) {
    std::copy(params, params + s->P, th.begin());
  } else {   // He-normal weights (Box-Muller on SplitMix64 draws), zero biases
    auto normal = [&](uint64_t k) {
      const double u1 = ((splitmix64(seed * 0x100000001b3ull + 2 * k) >> 11) + 1.0) / 9007199254740993.0;
      const double u2 = (splitmix64(seed * 0x100000001b3ull + 2 * k + 1) >> 11) / 9007199254740992.0;
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    };
    int64_t o = 0, k = 0;
    for (int64_t i = 0; i < (int64_t)H * kD; ++i) th[o++] = (float)(normal(k++) * std::sqrt(2.0 / kD));
    o += H;
    for (int64_t i = 0; i < (int64_t)H * H; ++i) th[o++] = (float)(normal(k++) * std::sqrt(2.0 / H));
    o += H;
    for (int64_t i = 0; i < H; ++i) th[o++] = (float)(normal(k++) * std::sqrt(1.0 / H));
  }
  if (cudaMalloc(&s->theta, s->P * 4) != cudaSuccess || cudaMalloc(&s->m, s->P * 4) != cudaSuccess ||
      cudaMalloc(&s->v, s->P * 4) != cudaSuccess || cudaMalloc(&s->W2b, (size_t)H * H * 2) != cudaSuccess) {
    cudaGetLastError();
    screen_free(s);
    return fail(TGBA_ENOMEM, "screen parameters");
  }
  TGBA_CUDA(cudaMemcpy(s->theta, th.data(), s->P * 4, cudaMemcpyHostToDevice));
  TGBA_CUDA(cudaMemset(s->m, 0, s->P * 4));
  TGBA_CUDA(cudaMemset(s->v, 0, s->P * 4));
  *out = s;
  return TGBA_OK;
}

void screen_free(Screen* s) {
  if (!s) return;
  if (s->theta) cudaFree(s->theta);
  if (s->m) cudaFree(s->m);
  if (s->v) cudaFree(s->v);
  if (s->W2b) cudaFree(s->W2b);
  delete s;
}

int64_t screen_nparams(const Screen* s) { return s->P; }

// Forward and backward of one batch; loss (mean squared error) into *loss, gradient into grad.
// work: float scratch of at least B * (4 H + 2) + 2 floats.
static tgba_status forward_backward(Screen& s, const float* x, const float* t, int64_t B, float* grad, float* work,
                                    double* d_loss, cudaStream_t st) {
  const int H = s.H;
  const float* W1 = s.theta;
  const float* b1 = W1 + (int64_t)H * kD;
  const float* W2 = b1 + H;
  const float* b2 = W2 + (int64_t)H * H;
  const float* w3 = b2 + H;
  const float* b3 = w3 + H;
  float* Z1 = work;
  float* H1 = Z1 + B * H;
  float* Z2 = H1 + B * H;
  float* H2 = Z2 + B * H;
  float* y = H2 + B * H;
  float* r = y + B;
  gemm<false, true>(st, (int)B, H, kD, x, W1, Z1);          // Z1 = X W1^T
  bias_relu<<<blocks(B * H), 256, 0, st>>>(B, H, Z1, b1, H1);
  gemm<false, true>(st, (int)B, H, H, H1, W2, Z2);          // Z2 = H1 W2^T
  bias_relu<<<blocks(B * H), 256, 0, st>>>(B, H, Z2, b2, H2);
  out_layer<<<blocks(B * 32), 256, 0, st>>>(B, H, H2, w3, b3, t, y, r);
  if (d_loss) {
    TGBA_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(double), st));
    sum_squares<<<blocks(B), 256, 0, st>>>(B, r, d_loss);
  }
  if (grad) {
    float* dW1 = grad;
    float* db1 = dW1 + (int64_t)H * kD;
    float* dW2 = db1 + H;
    float* db2 = dW2 + (int64_t)H * H;
    float* dw3 = db2 + H;
    float* db3 = dw3 + H;
    const float scale = 2.f / (float)B;                         // d(mean r^2)/dy = 2 r / B
    grad_out<<<(H + 1 + 127) / 128, 128, 0, st>>>(B, H, H2, r, scale, dw3, db3);
    float* dZ2 = H2;                                            // H2 is dead after grad_out
    back_out<<<blocks(B * H), 256, 0, st>>>(B, H, r, w3, Z2, scale, dZ2);
    gemm<true, false>(st, H, H, (int)B, dZ2, H1, dW2);          // dW2 = dZ2^T H1
    col_sum<<<(H + 127) / 128, 128, 0, st>>>(B, H, dZ2, 1.f, db2);
    float* dZ1 = Z2;                                            // Z2 is dead after back_out
    gemm<false, false>(st, (int)B, H, H, dZ2, W2, dZ1);         // dH1 = dZ2 W2
    relu_mask<<<blocks(B * H), 256, 0, st>>>(B * H, dZ1, Z1);   // dZ1 = dH1 * (Z1 > 0)
    gemm<true, false>(st, H, kD, (int)B, dZ1, x, dW1);          // dW1 = dZ1^T X
    col_sum<<<(H + 127) / 128, 128, 0, st>>>(B, H, dZ1, 1.f, db1);
  }
  TGBA_CUDA(cudaGetLastError());
  return TGBA_OK;
}

tgba_status screen_grad(Screen& s, const float* x, const float* t, int64_t B, float* grad, double* loss,
                        cudaStream_t st) {
  float* work = nullptr;
  double* d_loss = nullptr;
  TGBA_CUDA(cudaMallocAsync(&work, (size_t)(B * (4 * s.H + 2) + 2) * 4, st));
  TGBA_CUDA(cudaMallocAsync(&d_loss, sizeof(double), st));
  tgba_status r = forward_backward(s, x, t, B, grad, work, d_loss, st);
  double h = 0;
  if (r == TGBA_OK) {
    cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    *loss = h / (double)B;
  }
  cudaFreeAsync(work, st);
  cudaFreeAsync(d_loss, st);
  return r;
}

tgba_status screen_params(Screen& s, float* host) {
  TGBA_CUDA(cudaMemcpy(host, s.theta, s.P * 4, cudaMemcpyDeviceToHost));
  return TGBA_OK;
}

static tgba_status refresh_bf16(Screen& s, cudaStream_t st) {
  const float* W2 = s.theta + (int64_t)s.H * kD + s.H;
  to_bf16<<<blocks((int64_t)s.H * s.H), 256, 0, st>>>((int64_t)s.H * s.H, W2, s.W2b);
  TGBA_CUDA(cudaGetLastError());
  s.w2b_valid = true;
  return TGBA_OK;
}

// Layer-1 partials of every state of the basis (all sectors): part [n_ns_total + n_r_total][H],
// NS states first.  The caller frees *part (stream-ordered).
static tgba_status state_partials_all(Screen& s, Basis& b, float** part, cudaStream_t st) {
  const int H = s.H;
  const int64_t n_ns = (int64_t)b.ns.E.size(), n_r = (int64_t)b.r.E.size();
  TGBA_CUDA(cudaMallocAsync(part, (size_t)std::max<int64_t>(1, n_ns + n_r) * H * 4, st));
  const float* W1 = s.theta;
  const float* b1 = W1 + (int64_t)H * kD;
  if (n_ns > 0)
    state_partials<<<blocks(n_ns * H), 256, 0, st>>>(n_ns, true, b.d_modes_ns, b.d_M_ns, b.max_qp, b.d_nlab, b.L, H, W1,
                                                    b1, *part);
  if (n_r > 0)
    state_partials<<<blocks(n_r * H), 256, 0, st>>>(n_r, false, b.d_modes_r, b.d_M_r, b.max_qp, b.d_nlab, b.L, H, W1,
                                                   b1, *part + n_ns * H);
  TGBA_CUDA(cudaGetLastError());
  b.launches += 2;
  return TGBA_OK;
}

// Predicted y of every pair of sector `sidx`: pred float [n_ns][n_r].  Pairs outside the
// model (a state with more than Q quasiparticles) get 0.
tgba_status screen_score(Screen& s, Basis& b, int sidx, float* pred, cudaStream_t st) {
  if (s.H != 256) return fail(TGBA_EINVAL, "inference supports width 256");
  const Sector& sec = b.sectors[sidx];
  if (sec.n_ns == 0 || sec.n_r == 0) return TGBA_OK;
  if (!s.w2b_valid) {
    tgba_status r = refresh_bf16(s, st);
    if (r != TGBA_OK) return r;
  }
  std::vector<Rect> rects;
  for (const RectList& L : b.rect_lists)
    for (const Rect& rc : L.rects)
      if (rc.ns0 >= sec.ns_off && rc.ns0 < sec.ns_off + sec.n_ns) rects.push_back(rc);
  float* part = nullptr;
  tgba_status r = state_partials_all(s, b, &part, st);
  if (r != TGBA_OK) return r;
  const int H = s.H;
  const float* b2 = s.theta + (int64_t)H * kD + H + (int64_t)H * H;
  TGBA_CUDA(cudaMemsetAsync(pred, 0, (size_t)sec.n_ns * sec.n_r * 4, st));
  r = score_rects_tc(b, rects, part, part + (int64_t)b.ns.E.size() * H, s.W2b, b2, b2 + H, b2 + 2 * H, 0.f, 0.f,
                     pred, sec.x_off, nullptr, nullptr, nullptr, st);
  cudaFreeAsync(part, st);
  return r;
}

// The screened Pfaffian stage (after the contraction table): P = 0, the register-size pairs
// scored and the kept ones compacted into per-size lists, their Pfaffians from the lists, and
// the shared-memory sizes (n >= 16) without screening.  *kept: pairs evaluated by Pfaffian.
tgba_status screen_pfaffians(Screen& s, Basis& b, double tau, double hx, int64_t* kept, cudaStream_t st) {
  if (s.H != 256) return fail(TGBA_EINVAL, "inference supports width 256");
  if (!s.w2b_valid) {
    tgba_status r = refresh_bf16(s, st);
    if (r != TGBA_OK) return r;
  }
  const int H = s.H;
  constexpr int kSizes = 8;                                     // n = 0, 2, ..., 14
  std::vector<int64_t> off(kSizes + 1, 0);
  for (const Rect& rc : b.reg_rects) off[rc.n / 2 + 1] += (int64_t)rc.rows * rc.w;
  for (int i = 0; i < kSizes; ++i) off[i + 1] += off[i];
  TGBA_CUDA(cudaMemsetAsync(b.d_P, 0, (size_t)std::max<int64_t>(1, b.n_elements) * sizeof(double), st));
  void* lb = nullptr;
  const size_t list_bytes = (size_t)std::max<int64_t>(1, off[kSizes]) * sizeof(PairEntry);
  TGBA_CUDA(cudaMallocAsync(&lb, list_bytes + 64 * sizeof(int64_t), st));
  PairEntry* lists = (PairEntry*)lb;
  int64_t* d_off = (int64_t*)((char*)lb + list_bytes);
  unsigned* d_cnt = (unsigned*)(d_off + 16);
  TGBA_CUDA(cudaMemcpyAsync(d_off, off.data(), kSizes * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemsetAsync(d_cnt, 0, kSizes * sizeof(unsigned), st));
  float* part = nullptr;
  tgba_status r = state_partials_all(s, b, &part, st);
  if (r != TGBA_OK) { cudaFreeAsync(lb, st); return r; }
  const float* b2 = s.theta + (int64_t)H * kD + H + (int64_t)H * H;
  // keep iff y - (n/2) log10(L/24) + log10(L hx) >= log10(tau) - margin
  const float half_log_l = (float)(0.5 * std::log10(b.L / 24.0));
  const float shift = (float)(std::log10(b.L * std::fabs(hx)) - std::log10(tau) + s.margin);
  r = score_rects_tc(b, b.reg_rects, part, part + (int64_t)b.ns.E.size() * H, s.W2b, b2, b2 + H, b2 + 2 * H, shift,
                     half_log_l, nullptr, 0, d_cnt, d_off, lists, st);
  if (r == TGBA_OK) r = run_pfaffian_lists(b, d_cnt, d_off, lists, st);
  if (r == TGBA_OK) r = run_pfaffians_smem_classes(b, st);
  unsigned hc[kSizes] = {};
  if (r == TGBA_OK) {
    TGBA_CUDA(cudaMemcpyAsync(hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
  }
  cudaFreeAsync(part, st);
  cudaFreeAsync(lb, st);
  if (r != TGBA_OK) return r;
  TGBA_CUDA(cudaStreamSynchronize(st));
  int64_t k = b.n_elements - off[kSizes];                       // sizes n >= 16: all evaluated
  for (int i = 0; i < kSizes; ++i) k += hc[i];
  *kept = k;
  return TGBA_OK;
}

// Train on n_samples pairs drawn uniformly from all NS x R pairs of the given bases.
tgba_status screen_train(Basis** sets, int n_sets, int64_t n_samples, uint64_t seed, int H, int epochs, Screen** out,
                         double* stats, cudaStream_t st) {
  auto t_start = std::chrono::steady_clock::now();
  Screen* s = nullptr;
  tgba_status r = screen_create(H, nullptr, seed, &s);
  if (r != TGBA_OK) return r;
  // 1. sample: global element index -> (set, sector, a, b), grouped by (set, sector)
  std::vector<std::pair<int, int>> groups;
  std::vector<int64_t> cum;
  int64_t total = 0;
  for (int k = 0; k < n_sets; ++k)
    for (size_t q = 0; q < sets[k]->sectors.size(); ++q) {
      const Sector& sec = sets[k]->sectors[q];
      if (sec.n_ns * sec.n_r == 0) continue;
      groups.emplace_back(k, (int)q);
      cum.push_back(total);
      total += sec.n_ns * sec.n_r;
    }
  if (total == 0) { screen_free(s); return fail(TGBA_EINVAL, "training bases have no pairs"); }
  std::vector<std::vector<int32_t>> gp(groups.size());
  for (int64_t i = 0; i < n_samples; ++i) {
    const int64_t e = (int64_t)(splitmix64(seed ^ (0x5bd1e995ull * (uint64_t)(i + 1))) % (uint64_t)total);
    const size_t gi = std::upper_bound(cum.begin(), cum.end(), e) - cum.begin() - 1;
    const Sector& sec = sets[groups[gi].first]->sectors[groups[gi].second];
    const int64_t loc = e - cum[gi];
    gp[gi].push_back((int32_t)(loc / sec.n_r));
    gp[gi].push_back((int32_t)(loc % sec.n_r));
  }
  // 2. exact labels and features, group by group
  float *X = nullptr, *T = nullptr;
  TGBA_CUDA(cudaMalloc(&X, (size_t)n_samples * kD * 4));
  TGBA_CUDA(cudaMalloc(&T, (size_t)n_samples * 4));
  int64_t o = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const int64_t n = (int64_t)gp[gi].size() / 2;
    if (n == 0) continue;
    Basis& bb = *sets[groups[gi].first];
    const int sidx = groups[gi].second;
    const Sector& sec = bb.sectors[sidx];
    int32_t* dp = nullptr;
    double* dx = nullptr;
    TGBA_CUDA(cudaMalloc(&dp, n * 8));
    TGBA_CUDA(cudaMalloc(&dx, n * 16));
    TGBA_CUDA(cudaMemcpy(dp, gp[gi].data(), n * 8, cudaMemcpyHostToDevice));
    if (!bb.table_valid) {
      if ((r = build_table(bb, st)) != TGBA_OK) return r;
    }
    if ((r = run_pfaffian_pairs(bb, sidx, dp, n, dx, st)) != TGBA_OK) return r;
    pair_features<<<blocks(n), 256, 0, st>>>(n, dp, sec.ns_off, sec.r_off, bb.d_modes_ns, bb.d_modes_r, bb.d_M_ns,
                                             bb.d_M_r, bb.max_qp, bb.d_nlab, bb.L, X + o * kD);
    pair_targets<<<blocks(n), 256, 0, st>>>(n, dp, sec.ns_off, sec.r_off, bb.d_M_ns, bb.d_M_r, dx,
                                            std::log10(bb.L / 24.0), T + o);
    TGBA_CUDA(cudaGetLastError());
    TGBA_CUDA(cudaStreamSynchronize(st));
    cudaFree(dp);
    cudaFree(dx);
    o += n;
  }
  // 3. Adam on mini-batches; the last 5 % (in sample order) are held out for validation
  const int64_t n_val = std::max<int64_t>(1, n_samples / 20), n_tr = n_samples - n_val;
  const int64_t Bsz = 4096;
  float *work = nullptr, *grad = nullptr, *xb = nullptr, *tb = nullptr;
  int64_t* idx = nullptr;
  double* d_loss = nullptr;
  const int64_t wrows = std::max(Bsz, n_val);
  TGBA_CUDA(cudaMalloc(&work, (size_t)(wrows * (4 * H + 2) + 2) * 4));
  TGBA_CUDA(cudaMalloc(&grad, s->P * 4));
  TGBA_CUDA(cudaMalloc(&xb, Bsz * kD * 4));
  TGBA_CUDA(cudaMalloc(&tb, Bsz * 4));
  TGBA_CUDA(cudaMalloc(&idx, Bsz * 8));
  TGBA_CUDA(cudaMalloc(&d_loss, 8));
  std::vector<int64_t> perm(n_tr);
  std::iota(perm.begin(), perm.end(), 0);
  const float b1 = 0.9f, b2 = 0.999f;
  const int64_t steps_per_epoch = (n_tr + Bsz - 1) / Bsz;
  const int64_t total_steps = steps_per_epoch * epochs;
  double tr_sum = 0;
  int64_t tr_cnt = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t i = n_tr - 1; i > 0; --i) {          // Fisher-Yates with SplitMix64
      const int64_t j = (int64_t)(splitmix64(seed + 7919ull * (uint64_t)ep + 104729ull * (uint64_t)i) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    tr_sum = 0;
    tr_cnt = 0;
    for (int64_t k = 0; k < steps_per_epoch; ++k) {
      const int64_t bn = std::min(Bsz, n_tr - k * Bsz);
      TGBA_CUDA(cudaMemcpyAsync(idx, perm.data() + k * Bsz, bn * 8, cudaMemcpyHostToDevice, st));
      gather_rows<<<blocks(bn * kD), 256, 0, st>>>(bn, kD, idx, X, T, xb, tb);
      if ((r = forward_backward(*s, xb, tb, bn, grad, work, d_loss, st)) != TGBA_OK) return r;
      ++s->adam_step;
      // cosine-decayed learning rate from 2e-3
      const double frac = (double)(s->adam_step - 1) / std::max<int64_t>(1, total_steps);
      const float lr = (float)(2e-3 * 0.5 * (1.0 + std::cos(M_PI * frac)) + 1e-5);
      const float c1 = 1.f - std::pow(b1, (float)s->adam_step), c2 = 1.f - std::pow(b2, (float)s->adam_step);
      adam_kernel<<<blocks(s->P), 256, 0, st>>>(s->P, s->theta, grad, s->m, s->v, lr, b1, b2, c1, c2, 1e-8f);
      if (ep == epochs - 1) {
        double h = 0;
        TGBA_CUDA(cudaMemcpyAsync(&h, d_loss, 8, cudaMemcpyDeviceToHost, st));
        TGBA_CUDA(cudaStreamSynchronize(st));
        tr_sum += h;
        tr_cnt += bn;
      }
    }
  }
  TGBA_CUDA(cudaGetLastError());
  // validation RMSE -> margin (three standard errors)
  if ((r = forward_backward(*s, X + n_tr * kD, T + n_tr, n_val, nullptr, work, d_loss, st)) != TGBA_OK) return r;
  double vl = 0;
  TGBA_CUDA(cudaMemcpyAsync(&vl, d_loss, 8, cudaMemcpyDeviceToHost, st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  s->val_rmse = std::sqrt(vl / n_val);
  s->train_rmse = tr_cnt ? std::sqrt(tr_sum / tr_cnt) : 0;
  s->margin = 3.0 * s->val_rmse;
  cudaFree(X); cudaFree(T); cudaFree(work); cudaFree(grad); cudaFree(xb); cudaFree(tb); cudaFree(idx); cudaFree(d_loss);
  if ((r = refresh_bf16(*s, st)) != TGBA_OK) return r;
  TGBA_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    stats[0] = s->train_rmse;
    stats[1] = s->val_rmse;
    stats[2] = s->margin;
    stats[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  *out = s;
  return TGBA_OK;
}

}  // namespace tgba
