// Dense FP64 eigen-solver of the real-gauge H_eff (row a7; Eq. 1: diagonalising the truncated
// Hamiltonian gives E_a and M).  Library call: cuSOLVER's 64-bit syevd.
#include <cusolverDn.h>

#include <algorithm>
#include <cstdlib>
#include <string>
#include <thread>
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

struct EigWorker {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t params = nullptr;
  double* A = nullptr;
  int64_t a_cap = 0;
  void* work = nullptr;
  size_t work_cap = 0;
  std::vector<char> host;
  int* info = nullptr;
  int device = 0;
  tgba_status status = TGBA_OK;
  std::string msg;
};

struct EigPool {
  std::vector<EigWorker> w;
};

int pool_size() {
  const char* e = std::getenv("TGBA_EIG_WORKERS");
  int n = e ? std::atoi(e) : 8;
  return std::max(1, std::min(n, 32));
}

// One worker's share: build H~ of each sector, syevd (eigenvalues only) into evals.
void run_worker(Basis& b, EigWorker& w, const std::vector<int>& mine, double h_x, double* evals) {
  w.status = TGBA_OK;
  if (cudaSetDevice(w.device) != cudaSuccess) { w.status = TGBA_ECUDA; w.msg = "cudaSetDevice"; return; }
  for (int s : mine) {
    const Sector& sec = b.sectors[s];
    const int64_t n = sec.n_ns + sec.n_r;
    if (n * n > w.a_cap) {
      if (w.A) cudaFree(w.A);
      w.A = nullptr; w.a_cap = 0;
      if (cudaMalloc(&w.A, n * n * sizeof(double)) != cudaSuccess) { w.status = TGBA_ENOMEM; w.msg = "eigen-solver matrix"; return; }
      w.a_cap = n * n;
    }
    tgba_status r = build_real_heff(b, s, h_x, w.A, nullptr, sec.n_ns, nullptr, sec.n_r, w.st);
    if (r != TGBA_OK) { w.status = r; w.msg = "H_eff"; return; }
    size_t dev_bytes = 0, host_bytes = 0;
    cusolverStatus_t cs = cusolverDnXsyevd_bufferSize(w.h, w.params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                                      CUDA_R_64F, w.A, n, CUDA_R_64F, evals + sec.ev_off, CUDA_R_64F,
                                                      &dev_bytes, &host_bytes);
    if (cs != CUSOLVER_STATUS_SUCCESS) { w.status = TGBA_ECUDA; w.msg = "syevd buffer size"; return; }
    if (dev_bytes > w.work_cap) {
      if (w.work) cudaFree(w.work);
      w.work = nullptr; w.work_cap = 0;
      if (cudaMalloc(&w.work, dev_bytes) != cudaSuccess) { w.status = TGBA_ENOMEM; w.msg = "eigen-solver workspace"; return; }
      w.work_cap = dev_bytes;
    }
    if (w.host.size() < std::max<size_t>(1, host_bytes)) w.host.resize(std::max<size_t>(1, host_bytes));
    cs = cusolverDnXsyevd(w.h, w.params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, w.A, n,
                          CUDA_R_64F, evals + sec.ev_off, CUDA_R_64F, w.work, dev_bytes, w.host.data(), host_bytes,
                          w.info);
    if (cs != CUSOLVER_STATUS_SUCCESS) { w.status = TGBA_ECUDA; w.msg = "syevd"; return; }
    int info = 0;
    if (cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, w.st) != cudaSuccess ||
        cudaStreamSynchronize(w.st) != cudaSuccess) { w.status = TGBA_ECUDA; w.msg = "syevd info"; return; }
    if (info != 0) { w.status = TGBA_ENUMERIC; w.msg = "syevd did not converge"; return; }
  }
  if (cudaEventRecord(w.done, w.st) != cudaSuccess) { w.status = TGBA_ECUDA; w.msg = "event"; }
}

}  // namespace

void destroy_eig_pool(void* pool) {
  EigPool* p = (EigPool*)pool;
  for (EigWorker& w : p->w) {
    if (w.params) cusolverDnDestroyParams(w.params);
    if (w.h) cusolverDnDestroy(w.h);
    if (w.A) cudaFree(w.A);
    if (w.work) cudaFree(w.work);
    if (w.info) cudaFree(w.info);
    if (w.done) cudaEventDestroy(w.done);
    if (w.st) cudaStreamDestroy(w.st);
  }
  delete p;
}

tgba_status eig_all_sectors(Basis& b, double h_x, double* evals, cudaStream_t st) {
  EigPool* pool = (EigPool*)b.eig_pool;
  if (pool == nullptr) {
    pool = new EigPool();
    b.eig_pool = pool;
    pool->w.resize(pool_size());
    for (EigWorker& w : pool->w) {
      w.device = b.device;
      TGBA_CUDA(cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking));
      TGBA_CUDA(cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
      TGBA_CUDA(cudaMalloc(&w.info, sizeof(int)));
      if (cusolverDnCreate(&w.h) != CUSOLVER_STATUS_SUCCESS) return fail(TGBA_ECUDA, "cuSOLVER create");
      if (cusolverDnCreateParams(&w.params) != CUSOLVER_STATUS_SUCCESS) return fail(TGBA_ECUDA, "cuSOLVER params");
      cusolverDnSetStream(w.h, w.st);
    }
  }
  // longest-processing-time assignment of sectors (cost ~ n^3) to workers
  std::vector<int> order(b.sectors.size());
  for (size_t s = 0; s < order.size(); ++s) order[s] = (int)s;
  auto size = [&](int s) { return b.sectors[s].n_ns + b.sectors[s].n_r; };
  std::sort(order.begin(), order.end(), [&](int x, int y) { return size(x) > size(y); });
  const int W = (int)pool->w.size();
  std::vector<std::vector<int>> share(W);
  std::vector<double> load(W, 0.0);
  for (int s : order) {
    if (size(s) == 0) continue;
    int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    share[k].push_back(s);
    load[k] += (double)size(s) * size(s) * size(s);
  }
  cudaEvent_t ready;
  TGBA_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  TGBA_CUDA(cudaEventRecord(ready, st));
  for (EigWorker& w : pool->w) TGBA_CUDA(cudaStreamWaitEvent(w.st, ready, 0));
  std::vector<std::thread> threads;
  for (int k = 0; k < W; ++k)
    if (!share[k].empty()) threads.emplace_back(run_worker, std::ref(b), std::ref(pool->w[k]), std::cref(share[k]), h_x, evals);
  for (std::thread& t : threads) t.join();
  cudaEventDestroy(ready);
  for (int k = 0; k < W; ++k) {
    if (share[k].empty()) continue;
    EigWorker& w = pool->w[k];
    if (w.status != TGBA_OK) return fail(w.status, "eigen-solver worker: " + w.msg);
    TGBA_CUDA(cudaStreamWaitEvent(st, w.done, 0));
  }
  return TGBA_OK;
}

}  // namespace tgba
