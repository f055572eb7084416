// Dense FP64 eigen-solver of the real-gauge H_eff (row a7; Eq. 1: diagonalising the truncated
// Hamiltonian gives E_a and M).  Library call: cuSOLVER's 64-bit syevd.
#include <cusolverDn.h>

#include <string>

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
