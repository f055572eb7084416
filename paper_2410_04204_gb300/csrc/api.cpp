// The C ABI declared in include/tgba.h: argument checks, handle life cycle, device uploads,
// status words, and the order of the stages of each call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <set>
#include <string>

#include "tgba_internal.h"

namespace tgba {

static thread_local std::string g_last_error;

tgba_status fail(tgba_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

tgba_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TGBA_ENOMEM : TGBA_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

tgba_status check_status(Basis& b, cudaStream_t st) {
  unsigned w = 0;
  TGBA_CUDA(cudaMemcpyAsync(&w, b.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  if (w == 0) return TGBA_OK;
  TGBA_CUDA(cudaMemsetAsync(b.d_status, 0, sizeof(unsigned), st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  if (w & kStTimeout) return fail(TGBA_ETIMEOUT, "a bounded device wait gave up");
  if (w & kStBadIndex) return fail(TGBA_EINVAL, "a pair index was outside the sector");
  if (w & kStEigen) return fail(TGBA_ENUMERIC, "the eigen-solver met a non-finite matrix entry");
  if (w & kStTableSingular) return fail(TGBA_ENUMERIC, "the vacuum block of the contraction matrix is singular");
  if (w & kStTableImag) return fail(TGBA_ENUMERIC, "the gauge-rotated contraction table is not real");
  return fail(TGBA_ENUMERIC, "a Pfaffian produced NaN or Inf");
}

tgba_status scratch(Basis& b, int64_t doubles, double** out) {
  if (doubles > b.scratch_cap) {
    if (b.d_scratch) cudaFree(b.d_scratch);
    b.d_scratch = nullptr;
    b.scratch_cap = 0;
    cudaError_t e = cudaMalloc(&b.d_scratch, doubles * sizeof(double));
    if (e != cudaSuccess) { cudaGetLastError(); return fail(TGBA_ENOMEM, "device scratch of " + std::to_string(doubles * 8) + " bytes"); }
    b.scratch_cap = doubles;
  }
  *out = b.d_scratch;
  return TGBA_OK;
}

static void release(Basis* b) {
  void* ptrs[] = {b->d_E_ns, b->d_E_r, b->d_M_ns, b->d_M_r, b->d_sel_ns, b->d_sel_r, b->d_modes_ns, b->d_modes_r,
                  b->d_theta, b->d_nlab, b->d_table, b->d_c0, b->d_work, b->d_P, b->d_status,
                  b->d_eig_a, b->d_eig_w, b->d_eig_work, b->d_eig_info, b->d_scratch,
                  b->d_reg_rects, b->d_counter, b->d_blas_ws, b->d_emu_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int e = 0; e < 3; ++e) {
    if (b->ev[e]) cudaEventDestroy(b->ev[e]);
    if (b->eig_ev[e]) cudaEventDestroy(b->eig_ev[e]);
  }
  for (int e = 0; e < 2; ++e)
    if (b->q_ev[e]) cudaEventDestroy(b->q_ev[e]);
  for (RectList& L : b->rect_lists)
    if (L.d_rects) cudaFree(L.d_rects);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->solver) destroy_solver(b->solver);
  if (b->blas) destroy_blas(b->blas);
  delete b;
}

template <class T>
static tgba_status upload(T** dst, const T* src, size_t count, int64_t* counter) {
  size_t bytes = std::max<size_t>(1, count) * sizeof(T);
  TGBA_CUDA(cudaMalloc((void**)dst, bytes));
  if (count) TGBA_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  *counter += (int64_t)(count * sizeof(T));
  return TGBA_OK;
}

static tgba_status require_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(TGBA_ECUDA, "no usable CUDA device");
  }
  return TGBA_OK;
}

static tgba_status build(const tgba_model* model, const int32_t* sectors, int32_t n_sectors, const tgba_trunc* trunc,
                         Basis* b) {
  tgba_status r = enumerate_basis(*model, sectors, n_sectors, *trunc, *b);
  if (r != TGBA_OK) return r;
  TGBA_CUDA(cudaGetDevice(&b->device));
  const int L = b->L, q = b->max_qp;
  const size_t nns = b->ns.E.size(), nr = b->r.E.size();
  // table rows: NS mode i -> L-1-i (rows ascend as modes descend), R mode i -> L+i
  std::vector<uint8_t> sel_ns(std::max<size_t>(1, nns * q), 0), sel_r(std::max<size_t>(1, nr * q), 0);
  for (size_t s = 0; s < nns; ++s) {
    const int M = b->ns.M[s];
    for (int u = 0; u < M; ++u) sel_ns[s * q + u] = (uint8_t)(L - 1 - b->ns.modes[s * q + (M - 1 - u)]);
  }
  for (size_t s = 0; s < nr; ++s) {
    const int M = b->r.M[s];
    for (int u = 0; u < M; ++u) sel_r[s * q + u] = (uint8_t)(L + b->r.modes[s * q + u]);
  }
  if ((r = upload(&b->d_E_ns, b->ns.E.data(), nns, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_E_r, b->r.E.data(), nr, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_M_ns, b->ns.M.data(), nns, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_M_r, b->r.M.data(), nr, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_sel_ns, sel_ns.data(), nns * q, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_sel_r, sel_r.data(), nr * q, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_modes_ns, b->ns.modes.data(), nns * q, &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_modes_r, b->r.modes.data(), nr * q, &b->upload_bytes)) != TGBA_OK) return r;
  Modes mns = make_modes(L, 0, b->h), mr = make_modes(L, 1, b->h);
  std::vector<double> th(2 * L);
  std::vector<int> nl(2 * L);
  for (int i = 0; i < L; ++i) {
    th[i] = mns.theta[i]; th[L + i] = mr.theta[i];
    nl[i] = mns.nlab[i]; nl[L + i] = mr.nlab[i];
  }
  b->vac_norm = mns.norm * mr.norm;
  b->norm_ns = mns.norm;
  b->norm_r = mr.norm;
  if ((r = upload(&b->d_theta, th.data(), th.size(), &b->upload_bytes)) != TGBA_OK) return r;
  if ((r = upload(&b->d_nlab, nl.data(), nl.size(), &b->upload_bytes)) != TGBA_OK) return r;
  TGBA_CUDA(cudaMalloc((void**)&b->d_table, sizeof(double) * 4 * L * L));
  TGBA_CUDA(cudaMalloc((void**)&b->d_c0, sizeof(double) * 4));
  TGBA_CUDA(cudaMalloc((void**)&b->d_work, sizeof(double) * 2 * (16 * L * L + 4 * L + 1)));
  TGBA_CUDA(cudaMalloc((void**)&b->d_P, sizeof(double) * std::max<int64_t>(1, b->n_elements)));
  TGBA_CUDA(cudaMalloc((void**)&b->d_status, sizeof(unsigned)));
  TGBA_CUDA(cudaMemset(b->d_status, 0, sizeof(unsigned)));
  TGBA_CUDA(cudaMalloc((void**)&b->d_counter, sizeof(unsigned long long)));
  build_rects(*b);
  for (RectList& L : b->rect_lists) {
    for (const Rect& t : L.rects) {
      double f = 0;
      for (int m = t.n - 2; m >= 2; m -= 2) f += 2.0 * m * (m - 1) + m;   // F(n), real Parlett-Reid
      b->pf_flops += f * (double)t.rows * t.w;
    }
    if (!L.rects.empty() && (r = upload(&L.d_rects, L.rects.data(), L.rects.size(), &b->upload_bytes)) != TGBA_OK)
      return r;
  }
  if ((r = upload(&b->d_reg_rects, b->reg_rects.data(), b->reg_rects.size(), &b->upload_bytes)) != TGBA_OK) return r;
  for (int e = 0; e < 3; ++e) TGBA_CUDA(cudaEventCreate(&b->ev[e]));
  if ((r = plan_pfaffians(*b)) != TGBA_OK) return r;
  return TGBA_OK;
}

static tgba_status ensure_c0_host(Basis& b, cudaStream_t st) {
  if (b.c0_host_valid) return TGBA_OK;
  TGBA_CUDA(cudaMemcpyAsync(b.c0_host, b.d_c0, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  tgba_status r = check_status(b, st);     // synchronises
  if (r != TGBA_OK) {
    b.table_valid = false;
    return r;
  }
  b.c0_host_valid = true;
  return TGBA_OK;
}

static tgba_status ensure_table(Basis& b, cudaStream_t st) {
  if (!b.table_valid) {
    tgba_status r = build_table(b, st);
    if (r != TGBA_OK) return r;
    b.c0_host_valid = false;
  }
  return ensure_c0_host(b, st);
}

// The stage without screening: contraction table, then the Pfaffians.  The first call builds the
// table eagerly, runs the autotuner, then captures the stage (with its timing events) into a
// CUDA graph on a private stream; every call launches that graph on the caller's stream.
static tgba_status compute_x_graph(Basis& b, cudaStream_t st) {
  tgba_status r;
  if (!b.tuned) {
    if ((r = ensure_table(b, st)) != TGBA_OK) return r;
    if ((r = autotune_pfaffians(b, st)) != TGBA_OK) return r;
  }
  if (!b.graph_exec) {
    cudaStream_t cs;
    TGBA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int64_t before = b.launches.load();
    TGBA_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaEventRecordWithFlags(b.ev[0], cs, cudaEventRecordExternal);
    r = build_table(b, cs);
    if (r == TGBA_OK) {
      cudaEventRecordWithFlags(b.ev[1], cs, cudaEventRecordExternal);
      r = run_pfaffians(b, cs);
      cudaEventRecordWithFlags(b.ev[2], cs, cudaEventRecordExternal);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (r != TGBA_OK) { if (g) cudaGraphDestroy(g); return r; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b.graph = g;
    TGBA_CUDA(cudaGraphInstantiate(&b.graph_exec, b.graph, 0));
    b.graph_launches = b.launches.load() - before;
    b.launches -= b.graph_launches;        // counted when the graph runs
  }
  TGBA_CUDA(cudaGraphLaunch(b.graph_exec, st));
  b.launches += b.graph_launches;
  b.table_valid = true;
  b.c0_host_valid = false;
  b.ev_recorded = true;
  return TGBA_OK;
}

static tgba_status compute_x(Basis& b, Screen* screen, double tau, double hx, cudaStream_t st) {
  if (screen && !(tau > 0)) return fail(TGBA_EINVAL, "screening needs tau > 0");
  tgba_status r;
  if (!screen) {
    if ((r = compute_x_graph(b, st)) != TGBA_OK) return r;
  } else {
    if (!b.tuned) {
      if ((r = ensure_table(b, st)) != TGBA_OK) return r;
      if ((r = autotune_pfaffians(b, st)) != TGBA_OK) return r;
    }
    TGBA_CUDA(cudaEventRecord(b.ev[0], st));
    if ((r = build_table(b, st)) != TGBA_OK) return r;
    b.c0_host_valid = false;
    TGBA_CUDA(cudaEventRecord(b.ev[1], st));
    int64_t kept = 0;
    if ((r = screen_pfaffians(*screen, b, tau, hx, &kept, st)) != TGBA_OK) return r;
    TGBA_CUDA(cudaEventRecord(b.ev[2], st));
    b.ev_recorded = true;
    b.x_evaluated = kept;
    b.x_screened = b.n_elements - kept;
  }
  b.x_valid = true;
  b.x_screen = screen;
  b.x_tau = tau;
  if (!screen) {
    b.x_evaluated = b.n_elements;
    b.x_screened = 0;
  }
  return TGBA_OK;
}

}  // namespace tgba

using namespace tgba;

#define BASIS_OK(b)                                                   \
  do {                                                                \
    if ((b) == nullptr) return fail(TGBA_EINVAL, "null basis handle"); \
  } while (0)

extern "C" {

const char* tgba_last_error(void) { return g_last_error.c_str(); }

int32_t tgba_device_count(void) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

tgba_status tgba_build_basis(const tgba_model* model, const int32_t* sectors_m, int32_t n_sectors,
                             const tgba_trunc* trunc, tgba_basis* out) {
  g_last_error.clear();
  if (!model || !sectors_m || !trunc || !out) return fail(TGBA_EINVAL, "null argument");
  *out = nullptr;
  if (model->L < 4 || model->L > kMaxL || model->L % 2) return fail(TGBA_EINVAL, "L must be even, 4 <= L <= 120");
  if (!(model->J > 0) || !std::isfinite(model->J)) return fail(TGBA_EINVAL, "J must be positive");
  if (!(model->h_z > 0) || !std::isfinite(model->h_z)) return fail(TGBA_EINVAL, "h_z must be positive");
  if (n_sectors < 1 || n_sectors > model->L) return fail(TGBA_EINVAL, "need 1..L sectors");
  std::set<int> seen;
  for (int s = 0; s < n_sectors; ++s) {
    if (sectors_m[s] < 0 || sectors_m[s] >= model->L) return fail(TGBA_EINVAL, "sector m outside [0, L)");
    if (!seen.insert(sectors_m[s]).second) return fail(TGBA_EINVAL, "repeated sector");
  }
  if (trunc->max_qp < 0 || trunc->max_qp > kMaxQp) return fail(TGBA_EINVAL, "max_qp must be in [0, 16]");
  if (std::isnan(trunc->e_cut)) return fail(TGBA_EINVAL, "e_cut is NaN");
  tgba_status r = require_device();
  if (r != TGBA_OK) return r;
  Basis* b = new (std::nothrow) Basis();
  if (!b) return fail(TGBA_ENOMEM, "host allocation");
  r = build(model, sectors_m, n_sectors, trunc, b);
  if (r != TGBA_OK) {
    release(b);
    return r;
  }
  *out = (tgba_basis)b;
  return TGBA_OK;
}

tgba_status tgba_basis_info(tgba_basis h, int32_t s, int64_t* n_ns, int64_t* n_r, double* E0, uint8_t* parity,
                            uint8_t* nqp, int16_t* modes) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  const Sector& sec = b->sectors[s];
  if (n_ns) *n_ns = sec.n_ns;
  if (n_r) *n_r = sec.n_r;
  const int q = b->max_qp;
  for (int64_t i = 0; i < sec.n_ns + sec.n_r; ++i) {
    const bool ns = i < sec.n_ns;
    const StateTable& T = ns ? b->ns : b->r;
    const int64_t j = ns ? sec.ns_off + i : sec.r_off + (i - sec.n_ns);
    if (E0) E0[i] = T.E[j];
    if (parity) parity[i] = ns ? 0 : 1;
    if (nqp) nqp[i] = T.M[j];
    if (modes) std::memcpy(modes + i * q, T.modes.data() + j * q, q * sizeof(int16_t));
  }
  return TGBA_OK;
}

tgba_status tgba_basis_totals(tgba_basis h, int32_t* n_sectors, int64_t* n_elements, int64_t* n_heff) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (n_sectors) *n_sectors = (int32_t)b->sectors.size();
  if (n_elements) *n_elements = b->n_elements;
  if (n_heff) *n_heff = b->n_heff;
  return TGBA_OK;
}

tgba_status tgba_basis_free(tgba_basis h) {
  if (h) release((Basis*)h);
  return TGBA_OK;
}

tgba_status tgba_compute_x(tgba_basis h, tgba_screen screen, double tau, double screen_hx, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  return compute_x(*b, (Screen*)screen, tau, screen_hx, (cudaStream_t)stream);
}

tgba_status tgba_x_stats(tgba_basis h, int64_t* n_evaluated, int64_t* n_screened) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet");
  if (n_evaluated) *n_evaluated = b->x_evaluated;
  if (n_screened) *n_screened = b->x_screened;
  return TGBA_OK;
}

tgba_status tgba_x_export(tgba_basis h, int32_t s, double* x_dev, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  if (!x_dev && b->sectors[s].n_ns * b->sectors[s].n_r > 0) return fail(TGBA_EINVAL, "null output");
  return export_x(*b, s, x_dev, (cudaStream_t)stream);
}

tgba_status tgba_x_pairs(tgba_basis h, int32_t s, const int32_t* pairs_dev, int64_t n_pairs, double* out_dev,
                         void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (n_pairs < 0 || (n_pairs > 0 && (!pairs_dev || !out_dev))) return fail(TGBA_EINVAL, "bad pair list");
  cudaStream_t st = (cudaStream_t)stream;
  tgba_status r = ensure_table(*b, st);
  if (r != TGBA_OK) return r;
  if ((r = run_pfaffian_pairs(*b, s, pairs_dev, n_pairs, out_dev, st)) != TGBA_OK) return r;
  return check_status(*b, st);
}

tgba_status tgba_x_direct(tgba_basis h, int32_t s, const int32_t* pairs_dev, int64_t n_pairs, double* out_dev,
                          void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (n_pairs < 0 || (n_pairs > 0 && (!pairs_dev || !out_dev))) return fail(TGBA_EINVAL, "bad pair list");
  int limit = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
  if (x_direct_smem(b->L, b->max_qp, -1) + 16384 > (size_t)limit)
    return fail(TGBA_EINVAL, "the direct Pfaffian of size 2L + 2 max_qp does not fit in shared memory");
  cudaStream_t st = (cudaStream_t)stream;
  tgba_status r = x_direct(*b, s, pairs_dev, n_pairs, out_dev, st);
  if (r != TGBA_OK) return r;
  return check_status(*b, st);
}

tgba_status tgba_z_elements(tgba_basis h, int32_t s, int32_t parity, int32_t j, const int32_t* pairs_dev,
                            int64_t n_pairs, double* out_dev, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (parity != 0 && parity != 1) return fail(TGBA_EINVAL, "parity must be 0 (NS) or 1 (R)");
  if (j < 0 || j >= b->L) return fail(TGBA_EINVAL, "need 0 <= j < L");
  if (n_pairs < 0 || (n_pairs > 0 && (!pairs_dev || !out_dev))) return fail(TGBA_EINVAL, "bad pair list");
  int limit = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
  if (z_reduced_smem(b->max_qp, j) + 16384 > (size_t)limit)
    return fail(TGBA_EINVAL, "the Pfaffian of size 2 max_qp + 2j does not fit in shared memory");
  if (n_pairs == 0) return TGBA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nE = 2 * (int64_t)b->L + 2 * j;
  double* tab = nullptr;
  TGBA_CUDA(cudaMallocAsync((void**)&tab, (2 * nE * nE + 4) * sizeof(double), st));
  tgba_status r = z_table(*b, parity, j, tab, tab + 2 * nE * nE, st);
  if (r == TGBA_OK) r = z_reduced_elements(*b, s, parity, j, j, tab, tab + 2 * nE * nE, pairs_dev, n_pairs, out_dev, st);
  cudaFreeAsync(tab, st);
  if (r != TGBA_OK) return r;
  return check_status(*b, st);
}

tgba_status tgba_table(tgba_basis h, double* c0_host, double* table_dev, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  cudaStream_t st = (cudaStream_t)stream;
  tgba_status r = ensure_table(*b, st);
  if (r != TGBA_OK) return r;
  if (c0_host) { c0_host[0] = b->c0_host[0]; c0_host[1] = b->c0_host[1]; }
  if (table_dev)
    TGBA_CUDA(cudaMemcpyAsync(table_dev, b->d_table, sizeof(double) * 4 * b->L * b->L, cudaMemcpyDeviceToDevice, st));
  TGBA_CUDA(cudaStreamSynchronize(st));
  return TGBA_OK;
}

tgba_status tgba_assemble_heff(tgba_basis h, double h_x, tgba_screen screen, double tau, double* heff_dev,
                               void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (!std::isfinite(h_x)) return fail(TGBA_EINVAL, "h_x must be finite");
  if (!heff_dev && b->n_heff > 0) return fail(TGBA_EINVAL, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->x_valid || b->x_screen != (const void*)screen || (screen && b->x_tau != tau)) {
    tgba_status r = compute_x(*b, (Screen*)screen, tau, h_x, st);
    if (r != TGBA_OK) return r;
  }
  return assemble_heff(*b, h_x, heff_dev, st);
}

tgba_status tgba_eigvals(tgba_basis h, const double* h_x, int32_t n_hx, double* evals_dev, void* stream) {
  return tgba_eigvals_ex(h, h_x, n_hx, 0, evals_dev, stream);
}

tgba_status tgba_eigvals_ex(tgba_basis h, const double* h_x, int32_t n_hx, int32_t method, double* evals_dev,
                            void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (method < 0 || method > 2) return fail(TGBA_EINVAL, "method must be 0 (automatic), 1 (native) or 2 (cuSOLVER)");
  if (!h_x || n_hx < 1) return fail(TGBA_EINVAL, "need at least one h_x");
  for (int i = 0; i < n_hx; ++i)
    if (!std::isfinite(h_x[i])) return fail(TGBA_EINVAL, "h_x must be finite");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  if (!evals_dev && b->n_states > 0) return fail(TGBA_EINVAL, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  tgba_status r = eig_all_sectors(*b, h_x, n_hx, evals_dev, method, st);
  if (r != TGBA_OK) return r;
  return check_status(*b, st);
}

tgba_status tgba_eigvals_wait_check(tgba_basis h, const double* h_x, int32_t n_hx, uint32_t spin_limit,
                                    int32_t withhold_matrix, int32_t withhold_rank, double* evals_dev, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (!h_x || n_hx < 1) return fail(TGBA_EINVAL, "need at least one h_x");
  for (int i = 0; i < n_hx; ++i)
    if (!std::isfinite(h_x[i])) return fail(TGBA_EINVAL, "h_x must be finite");
  if (spin_limit < 1) return fail(TGBA_EINVAL, "spin_limit must be at least 1");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  if (!evals_dev && b->n_states > 0) return fail(TGBA_EINVAL, "null output");
  int64_t n_max = 0;
  for (const Sector& s : b->sectors) n_max = std::max(n_max, s.n_ns + s.n_r);
  if ((n_max + 31) / 32 * 32 > kMaxNativeLd)
    return fail(TGBA_EINVAL, "the native eigen-solver takes sectors of at most " + std::to_string(kMaxNativeLd) + " states");
  cudaStream_t st = (cudaStream_t)stream;
  const WaitCheck check{spin_limit, withhold_matrix, withhold_rank};
  tgba_status r = eig_all_sectors_native(*b, h_x, n_hx, evals_dev, st, &check);
  if (r != TGBA_OK) return r;
  return check_status(*b, st);
}

tgba_status tgba_dsf(tgba_basis h, int32_t s, double h_x, double w_min, double w_max, int32_t n_w, double eta,
                     float* S_dev, double* evals_dev, int32_t n_ev, double* weights_dev, double* dE_dev,
                     void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (b->sectors[s].m != 0) return fail(TGBA_EINVAL, "S(k=0, w) needs the k = 0 sector");
  if (n_w < 1 || !S_dev) return fail(TGBA_EINVAL, "need n_w >= 1 and an output buffer");
  if (!(eta > 0) || !std::isfinite(w_min) || !std::isfinite(w_max) || !std::isfinite(h_x))
    return fail(TGBA_EINVAL, "eta must be positive and the grid finite");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  return dsf(*b, s, h_x, w_min, w_max, n_w, eta, S_dev, evals_dev, n_ev, weights_dev, dE_dev, (cudaStream_t)stream);
}

tgba_status tgba_dsf_k(tgba_basis h, int32_t s, int32_t s0, double h_x, double w_min, double w_max, int32_t n_w,
                       double eta, float* S_dev, double* evals_dev, int32_t n_ev, double* weights_dev, double* dE_dev,
                       void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  const int ns = (int)b->sectors.size();
  if (s < 0 || s >= ns || s0 < 0 || s0 >= ns) return fail(TGBA_EINVAL, "sector index out of range");
  if (b->sectors[s0].m != 0) return fail(TGBA_EINVAL, "s0 must be the k = 0 sector (it holds the ground state)");
  if (n_w < 1 || !S_dev) return fail(TGBA_EINVAL, "need n_w >= 1 and an output buffer");
  if (!(eta > 0) || !std::isfinite(w_min) || !std::isfinite(w_max) || !std::isfinite(h_x))
    return fail(TGBA_EINVAL, "eta must be positive and the grid finite");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  cudaStream_t st = (cudaStream_t)stream;
  tgba_status r = ensure_table(*b, st);
  if (r != TGBA_OK) return r;
  return dsf_k(*b, s, s0, h_x, w_min, w_max, n_w, eta, S_dev, evals_dev, n_ev, weights_dev, dE_dev, st);
}

tgba_status tgba_quench(tgba_basis h, int32_t s, double h_z0, const double* hx_variants, const double* ecut_variants,
                        int32_t n_variants, double t_max, int32_t n_t, int32_t method, double* mx_dev, double* norm_dev,
                        int64_t* chi_host, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (b->sectors[s].m != 0) return fail(TGBA_EINVAL, "the quench needs the k = 0 sector");
  if (n_variants < 1 || !hx_variants || !ecut_variants || !mx_dev || n_t < 1)
    return fail(TGBA_EINVAL, "need variants, n_t >= 1 and an output buffer");
  if (!(h_z0 > 0) || !std::isfinite(t_max) || t_max < 0) return fail(TGBA_EINVAL, "need h_z0 > 0 and t_max >= 0");
  if (method < 0 || method > 2) return fail(TGBA_EINVAL, "method must be 0 (automatic), 1 (eigen) or 2 (Chebyshev)");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  tgba_status r = ensure_c0_host(*b, (cudaStream_t)stream);
  if (r != TGBA_OK) return r;
  return quench(*b, s, h_z0, hx_variants, ecut_variants, n_variants, 0, t_max, n_t, method, mx_dev, norm_dev, nullptr,
                chi_host, (cudaStream_t)stream);
}

tgba_status tgba_quench_ordered(tgba_basis h, int32_t s, double h_z0, const double* hx_variants,
                                const double* trunc_variants, int32_t n_variants, int32_t order, double t_max,
                                int32_t n_t, int32_t method, double* mx_dev, double* norm_dev, double* eps_dev,
                                int64_t* chi_host, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (b->sectors[s].m != 0) return fail(TGBA_EINVAL, "the quench needs the k = 0 sector");
  if (n_variants < 1 || !hx_variants || !trunc_variants || !mx_dev || n_t < 1)
    return fail(TGBA_EINVAL, "need variants, n_t >= 1 and an output buffer");
  if (!(h_z0 > 0) || !std::isfinite(t_max) || t_max < 0) return fail(TGBA_EINVAL, "need h_z0 > 0 and t_max >= 0");
  if (method < 0 || method > 2) return fail(TGBA_EINVAL, "method must be 0 (automatic), 1 (eigen) or 2 (Chebyshev)");
  if (order != 0 && order != 1) return fail(TGBA_EINVAL, "order must be 0 (energy) or 1 (overlap)");
  for (int v = 0; v < n_variants; ++v) {
    if (!std::isfinite(hx_variants[v]) || !std::isfinite(trunc_variants[v])) return fail(TGBA_EINVAL, "non-finite variant");
    if (order == 1 && !(trunc_variants[v] >= 1 && trunc_variants[v] == std::floor(trunc_variants[v])))
      return fail(TGBA_EINVAL, "with order 1 each variant is a whole number of states >= 1");
  }
  if (eps_dev)
    for (int v = 0; v + 1 < n_variants; ++v) {
      const double a = trunc_variants[v], c = trunc_variants[v + 1];
      const bool nested = order == 1 ? a <= c : (c < 0 || (a >= 0 && a <= c));
      if (!nested) return fail(TGBA_EINVAL, "the convergence metric needs nested variants (non-decreasing truncation)");
    }
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  tgba_status r = ensure_c0_host(*b, (cudaStream_t)stream);
  if (r != TGBA_OK) return r;
  return quench(*b, s, h_z0, hx_variants, trunc_variants, n_variants, order, t_max, n_t, method, mx_dev, norm_dev,
                eps_dev, chi_host, (cudaStream_t)stream);
}

tgba_status tgba_quench_correlators(tgba_basis h, int32_t s, double h_z0, double h_x, double trunc, int32_t order,
                                   double t_max, int32_t n_t, int32_t j_max, double* mx_dev, double* corr_dev,
                                   double* norm_dev, int64_t* chi_host, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (s < 0 || s >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  if (b->sectors[s].m != 0) return fail(TGBA_EINVAL, "the quench needs the k = 0 sector");
  if (!mx_dev || !corr_dev || n_t < 1 || j_max < 1 || j_max >= b->L)
    return fail(TGBA_EINVAL, "need output buffers, n_t >= 1 and 1 <= j_max < L");
  if (!(h_z0 > 0) || !std::isfinite(t_max) || t_max < 0 || !std::isfinite(h_x) || !std::isfinite(trunc))
    return fail(TGBA_EINVAL, "need h_z0 > 0, t_max >= 0 and finite fields");
  if (order != 0 && order != 1) return fail(TGBA_EINVAL, "order must be 0 (energy) or 1 (overlap)");
  if (order == 1 && !(trunc >= 1 && trunc == std::floor(trunc)))
    return fail(TGBA_EINVAL, "with order 1 the truncation is a whole number of states >= 1");
  int limit = 0;
  TGBA_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
  if (z_reduced_smem(b->max_qp, j_max) + 16384 > (size_t)limit)
    return fail(TGBA_EINVAL, "the Pfaffian of size 2 max_qp + 2 j_max does not fit in shared memory");
  if (!b->x_valid) return fail(TGBA_EINVAL, "no X computed yet: call tgba_compute_x");
  tgba_status r = ensure_c0_host(*b, (cudaStream_t)stream);
  if (r != TGBA_OK) return r;
  return quench(*b, s, h_z0, &h_x, &trunc, 1, order, t_max, n_t, 1, mx_dev, norm_dev, nullptr, chi_host,
                (cudaStream_t)stream, j_max, corr_dev);
}

tgba_status tgba_screen_create(int32_t width, const float* params_host, uint64_t seed, tgba_screen* out) {
  if (!out || width != 256) return fail(TGBA_EINVAL, "width must be 256 and out non-null");
  tgba_status r = require_device();
  if (r != TGBA_OK) return r;
  Screen* s = nullptr;
  if ((r = screen_create(width, params_host, seed, &s)) != TGBA_OK) return r;
  *out = (tgba_screen)s;
  return TGBA_OK;
}

tgba_status tgba_screen_nparams(tgba_screen s, int64_t* n) {
  if (!s || !n) return fail(TGBA_EINVAL, "null argument");
  *n = screen_nparams((Screen*)s);
  return TGBA_OK;
}

tgba_status tgba_screen_params(tgba_screen s, float* params_host) {
  if (!s || !params_host) return fail(TGBA_EINVAL, "null argument");
  return screen_params(*(Screen*)s, params_host);
}

tgba_status tgba_screen_grad(tgba_screen s, const float* x_dev, const float* t_dev, int64_t B, float* grad_dev,
                             double* loss_host, void* stream) {
  if (!s || !x_dev || !t_dev || !grad_dev || !loss_host || B < 1) return fail(TGBA_EINVAL, "bad arguments");
  return screen_grad(*(Screen*)s, x_dev, t_dev, B, grad_dev, loss_host, (cudaStream_t)stream);
}

tgba_status tgba_screen_train(const tgba_basis* sets, int32_t n_sets, int64_t n_samples, uint64_t seed, int32_t width,
                              int32_t epochs, tgba_screen* out, double* stats_host, void* stream) {
  if (!sets || n_sets < 1 || n_samples < 20 || epochs < 1 || width != 256 || !out)
    return fail(TGBA_EINVAL, "need bases, n_samples >= 20, epochs >= 1, width 256");
  std::vector<Basis*> v;
  for (int i = 0; i < n_sets; ++i) {
    if (!sets[i]) return fail(TGBA_EINVAL, "null basis handle");
    v.push_back((Basis*)sets[i]);
  }
  Screen* s = nullptr;
  tgba_status r = screen_train(v.data(), n_sets, n_samples, seed, width, epochs, &s, stats_host, (cudaStream_t)stream);
  if (r != TGBA_OK) return r;
  *out = (tgba_screen)s;
  return TGBA_OK;
}

tgba_status tgba_screen_predict(tgba_screen s, tgba_basis h, int32_t sector, float* pred_dev, void* stream) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (!s || !pred_dev) return fail(TGBA_EINVAL, "null argument");
  if (sector < 0 || sector >= (int)b->sectors.size()) return fail(TGBA_EINVAL, "sector index out of range");
  return screen_score(*(Screen*)s, *b, sector, pred_dev, (cudaStream_t)stream);
}

tgba_status tgba_screen_free(tgba_screen s) {
  screen_free((Screen*)s);
  return TGBA_OK;
}

tgba_status tgba_profile(tgba_basis h, tgba_prof* out) {
  Basis* b = (Basis*)h;
  BASIS_OK(b);
  if (!out) return fail(TGBA_EINVAL, "null output");
  std::memset(out, 0, sizeof(*out));
  if (b->ev_recorded) {
    float t0 = 0, t1 = 0;
    TGBA_CUDA(cudaEventSynchronize(b->ev[2]));
    TGBA_CUDA(cudaEventElapsedTime(&t0, b->ev[0], b->ev[1]));
    TGBA_CUDA(cudaEventElapsedTime(&t1, b->ev[1], b->ev[2]));
    out->table_ms = t0;
    out->pfaffian_ms = t1;
  }
  out->pfaffian_flops = b->pf_flops;
  out->pfaffian_launches = (int64_t)b->pf_plan.size();
  out->kernel_launches = b->launches.load();
  out->upload_bytes = b->upload_bytes;
  out->evaluated = b->x_evaluated;
  out->tune_mode = b->tuned ? b->tune_mode : -1;
  out->tune_threads = b->tune_threads;
  for (size_t i = 0; i < b->tune_log.size() && i < 8; ++i) out->tune_ms[i] = b->tune_log[i].ms;
  if (b->eig_ev_recorded) {
    float t0 = 0, t1 = 0;
    TGBA_CUDA(cudaEventSynchronize(b->eig_ev[2]));
    TGBA_CUDA(cudaEventElapsedTime(&t0, b->eig_ev[0], b->eig_ev[1]));
    TGBA_CUDA(cudaEventElapsedTime(&t1, b->eig_ev[1], b->eig_ev[2]));
    out->tridiag_ms = t0;
    out->bisect_ms = t1;
  }
  out->tridiag_flops = b->tridiag_flops;
  out->eig_matrices = b->eig_matrices;
  if (b->q_ev_recorded) {
    float t = 0;
    TGBA_CUDA(cudaEventSynchronize(b->q_ev[1]));
    TGBA_CUDA(cudaEventElapsedTime(&t, b->q_ev[0], b->q_ev[1]));
    out->quench_ms = t;
  }
  out->quench_flops = b->quench_flops;
  out->quench_terms = b->quench_terms;
  out->quench_prep_ms = b->quench_prep_ms;
  out->quench_gram_ms = b->quench_gram_ms;
  out->quench_eval_ms = b->quench_eval_ms;
  out->eig_cluster = b->eig_cluster;
  return TGBA_OK;
}

tgba_status tgba_fp64_peak(int32_t reps, double* gflops) {
  if (!gflops || reps < 1) return fail(TGBA_EINVAL, "bad arguments");
  tgba_status r = require_device();
  if (r != TGBA_OK) return r;
  return fp64_peak(reps, gflops);
}

}  // extern "C"
