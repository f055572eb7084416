// Dense FP64 eigen-solver of the real-gauge H_eff (row a7; Eq. 1: diagonalising the truncated
// Hamiltonian gives E_a and M), library path: cuSOLVER's 64-bit syevd with eigenvectors (DSF,
// quench) and its batched XsyevBatched for eigenvalues of sectors too large for the native
// solver in tridiag.cu.
#include <cusolverDn.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "tgba_internal.h"

namespace tgba {

void destroy_solver(void* h) { cusolverDnDestroy((cusolverDnHandle_t)h); }

static tgba_status solver_fail(cusolverStatus_t s, const char* what) {
  return fail(TGBA_ECUDA, std::string("cuSOLVER ") + what + " failed with status " + std::to_string((int)s));
}

tgba_status eig_sym(Basis& b, int64_t n, double* a, double* w, bool vectors, cudaStream_t st) {
  if (n == 0) return TGBA_OK;
  cusolverDnHandle_t h = (cusolverDnHandle_t)b.solver;
  if (h == nullptr) {
    cusolverStatus_t s = cusolverDnCreate(&h);
    if (s != CUSOLVER_STATUS_SUCCESS) return solver_fail(s, "create");
    b.solver = h;
  }
  cusolverDnSetStream(h, st);
  cusolverDnParams_t params;
  cusolverStatus_t s = cusolverDnCreateParams(&params);
  if (s != CUSOLVER_STATUS_SUCCESS) return solver_fail(s, "params");
  const cusolverEigMode_t jobz = vectors ? CUSOLVER_EIG_MODE_VECTOR : CUSOLVER_EIG_MODE_NOVECTOR;
  size_t dev_bytes = 0, host_bytes = 0;
  s = cusolverDnXsyevd_bufferSize(h, params, jobz, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, a, n, CUDA_R_64F, w,
                                  CUDA_R_64F, &dev_bytes, &host_bytes);
  if (s != CUSOLVER_STATUS_SUCCESS) { cusolverDnDestroyParams(params); return solver_fail(s, "syevd buffer"); }
  if ((int64_t)dev_bytes > b.eig_work_cap) {
    if (b.d_eig_work) cudaFree(b.d_eig_work);
    b.d_eig_work = nullptr;
    b.eig_work_cap = 0;
    cudaError_t e = cudaMalloc(&b.d_eig_work, dev_bytes);
    if (e != cudaSuccess) { cusolverDnDestroyParams(params); return fail(TGBA_ENOMEM, "eigen-solver workspace"); }
    b.eig_work_cap = (int64_t)dev_bytes;
  }
  if (b.d_eig_info == nullptr) {
    cudaError_t e = cudaMalloc(&b.d_eig_info, sizeof(int));
    if (e != cudaSuccess) { cusolverDnDestroyParams(params); return fail(TGBA_ENOMEM, "eigen-solver info"); }
  }
  std::vector<char> host_work(host_bytes > 0 ? host_bytes : 1);
  s = cusolverDnXsyevd(h, params, jobz, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, a, n, CUDA_R_64F, w, CUDA_R_64F,
                       b.d_eig_work, dev_bytes, host_work.data(), host_bytes, b.d_eig_info);
  cusolverDnDestroyParams(params);
  if (s != CUSOLVER_STATUS_SUCCESS) return solver_fail(s, "syevd");
  int info = 0;
  TGBA_CUDA(cudaMemcpyAsync(&info, b.d_eig_info, sizeof(int), cudaMemcpyDeviceToHost, st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  if (info != 0) return fail(TGBA_ENUMERIC, "syevd did not converge (info " + std::to_string(info) + ")");
  return TGBA_OK;
}

}  // namespace tgba

namespace tgba {
namespace {

// Slot q of the batch holds sector s at field hx[h]: its real-gauge H~ (n_s x n_s) in the
// top-left corner of an n_max x n_max matrix, zeros elsewhere.
__global__ void heff_real_padded(int64_t kn, int64_t kr, int64_t n_max, int64_t n_r, const double* __restrict__ E_ns,
                                 const double* __restrict__ E_r, const double* __restrict__ P,
                                 const double* __restrict__ c0, double scale, double* __restrict__ A) {
  const int64_t n = kn + kr;
  const double c = scale * sqrt(c0[0] * c0[0] + c0[1] * c0[1]);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_max * n_max;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = idx / n_max, row = idx - col * n_max;
    double v = 0.0;
    if (row < n && col < n) {
      if (row == col) v = row < kn ? E_ns[row] : E_r[row - kn];
      else if (row < kn && col >= kn) v = c * P[row * n_r + (col - kn)];
      else if (row >= kn && col < kn) v = c * P[col * n_r + (row - kn)];
    }
    A[idx] = v;
  }
}

// Order-preserving map of doubles onto unsigned integers (and back), for atomicMax.
__device__ __forceinline__ unsigned long long ordered(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unordered(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Gershgorin upper bound of each slot's spectrum: thread = row of the n x n corner
// (column-major reads are coalesced across the warp), block maximum, atomicMax per slot.
__global__ void gershgorin_kernel(const int64_t* __restrict__ nq, int64_t n_max, const double* __restrict__ A,
                                  unsigned long long* __restrict__ bound) {
  __shared__ double red[32];
  const int64_t q = blockIdx.y, n = nq[q];
  const double* Aq = A + q * n_max * n_max;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double r = -1e300;
  if (i < n) {
    r = Aq[i * n_max + i];
    for (int64_t j = 0; j < n; ++j)
      if (j != i) r += fabs(Aq[j * n_max + i]);
  }
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    atomicMax(bound + q, ordered(m));
  }
}

// Padding diagonal entries just above the bound, so the n true eigenvalues are the n smallest.
__global__ void pad_kernel(const int64_t* __restrict__ nq, int64_t n_max, const unsigned long long* __restrict__ bound,
                           double* __restrict__ A) {
  const int64_t q = blockIdx.y, n = nq[q];
  const double pad = unordered(bound[q]) + 1.0;
  for (int64_t i = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_max; i += (int64_t)gridDim.x * blockDim.x)
    A[q * n_max * n_max + i * n_max + i] = pad;
}

}  // namespace

static tgba_status eig_all_sectors_lib(Basis& b, const double* hx, int n_hx, double* evals, cudaStream_t st);

tgba_status eig_all_sectors(Basis& b, const double* hx, int n_hx, double* evals, int method, cudaStream_t st) {
  int64_t n_max = 0;
  for (const Sector& s : b.sectors) n_max = std::max(n_max, s.n_ns + s.n_r);
  const bool fits = (n_max + 31) / 32 * 32 <= kMaxNativeLd;
  if (method == 1 && !fits)
    return fail(TGBA_EINVAL, "the native eigen-solver takes sectors of at most " + std::to_string(kMaxNativeLd) + " states");
  if (method == 1 || (method == 0 && fits)) return eig_all_sectors_native(b, hx, n_hx, evals, st);
  return eig_all_sectors_lib(b, hx, n_hx, evals, st);
}

static tgba_status eig_all_sectors_lib(Basis& b, const double* hx, int n_hx, double* evals, cudaStream_t st) {
  int64_t n_max = 0;
  std::vector<std::pair<int, int>> slots;     // (h index, sector)
  for (int h = 0; h < n_hx; ++h)
    for (size_t s = 0; s < b.sectors.size(); ++s) {
      const int64_t n = b.sectors[s].n_ns + b.sectors[s].n_r;
      if (n == 0) continue;
      n_max = std::max(n_max, n);
      slots.emplace_back(h, (int)s);
    }
  if (slots.empty()) return TGBA_OK;
  const int64_t B = (int64_t)slots.size();
  double* A;
  tgba_status r = scratch(b, B * n_max * n_max + B * n_max + 3 * B + 2, &A);
  if (r != TGBA_OK) return r;
  double* W = A + B * n_max * n_max;
  int64_t* nq = (int64_t*)(W + B * n_max);
  unsigned long long* bound = (unsigned long long*)(nq + B);
  int* info = (int*)(bound + B);
  std::vector<int64_t> hn(B);
  for (int64_t q = 0; q < B; ++q) hn[q] = b.sectors[slots[q].second].n_ns + b.sectors[slots[q].second].n_r;
  TGBA_CUDA(cudaMemcpyAsync(nq, hn.data(), B * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  TGBA_CUDA(cudaMemsetAsync(bound, 0, B * sizeof(unsigned long long), st));
  for (int64_t q = 0; q < B; ++q) {
    const Sector& sec = b.sectors[slots[q].second];
    double* Aq = A + q * n_max * n_max;
    const int64_t work = n_max * n_max;
    const int grid = (int)std::min<int64_t>((work + 255) / 256, 152 * 32);
    heff_real_padded<<<grid, 256, 0, st>>>(sec.n_ns, sec.n_r, n_max, sec.n_r, b.d_E_ns + sec.ns_off,
                                          b.d_E_r + sec.r_off, b.d_P + sec.x_off, b.d_c0, -b.L * hx[slots[q].first], Aq);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
  }
  gershgorin_kernel<<<dim3((unsigned)((n_max + 255) / 256), (unsigned)B), 256, 0, st>>>(nq, n_max, A, bound);
  pad_kernel<<<dim3(4, (unsigned)B), 256, 0, st>>>(nq, n_max, bound, A);
  TGBA_CUDA(cudaGetLastError());
  b.launches += 2;
  cusolverDnHandle_t h = (cusolverDnHandle_t)b.solver;
  if (h == nullptr) {
    cusolverStatus_t cs = cusolverDnCreate(&h);
    if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail(cs, "create");
    b.solver = h;
  }
  cusolverDnSetStream(h, st);
  cusolverDnParams_t params;
  cusolverStatus_t cs = cusolverDnCreateParams(&params);
  if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail(cs, "params");
  size_t dev_bytes = 0, host_bytes = 0;
  cs = cusolverDnXsyevBatched_bufferSize(h, params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n_max,
                                         CUDA_R_64F, A, n_max, CUDA_R_64F, W, CUDA_R_64F, &dev_bytes, &host_bytes, B);
  if (cs != CUSOLVER_STATUS_SUCCESS) { cusolverDnDestroyParams(params); return solver_fail(cs, "syevBatched buffer"); }
  if ((int64_t)dev_bytes > b.eig_work_cap) {
    if (b.d_eig_work) cudaFree(b.d_eig_work);
    b.d_eig_work = nullptr;
    b.eig_work_cap = 0;
    if (cudaMalloc(&b.d_eig_work, dev_bytes) != cudaSuccess) {
      cudaGetLastError();
      cusolverDnDestroyParams(params);
      return fail(TGBA_ENOMEM, "batched eigen-solver workspace");
    }
    b.eig_work_cap = (int64_t)dev_bytes;
  }
  std::vector<char> host_work(std::max<size_t>(1, host_bytes));
  cs = cusolverDnXsyevBatched(h, params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n_max, CUDA_R_64F, A,
                              n_max, CUDA_R_64F, W, CUDA_R_64F, b.d_eig_work, dev_bytes, host_work.data(), host_bytes,
                              info, B);
  cusolverDnDestroyParams(params);
  if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail(cs, "syevBatched");
  std::vector<int> hinfo(B);
  TGBA_CUDA(cudaMemcpyAsync(hinfo.data(), info, B * sizeof(int), cudaMemcpyDeviceToHost, st));
  for (int64_t q = 0; q < B; ++q) {
    const Sector& sec = b.sectors[slots[q].second];
    TGBA_CUDA(cudaMemcpyAsync(evals + (int64_t)slots[q].first * b.n_states + sec.ev_off, W + q * n_max,
                              (sec.n_ns + sec.n_r) * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  TGBA_CUDA(cudaStreamSynchronize(st));
  for (int64_t q = 0; q < B; ++q)
    if (hinfo[q] != 0) return fail(TGBA_ENUMERIC, "batched eigen-solver did not converge (info " + std::to_string(hinfo[q]) + ")");
  return TGBA_OK;
}

}  // namespace tgba
