// Internal declarations shared by the translation units of libtgba.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tgba.h"

namespace tgba {

constexpr int kMaxQp = 16;        // quasiparticles per state
constexpr int kMaxL = 120;        // 2L excitation operators must index a uint8 table row
constexpr int kMaxN = 2 * kMaxQp; // largest Pfaffian M_a + M_b
constexpr int kNumClasses = 12;   // Pfaffian size classes (basis.cpp: tile_class)

// Device status word bits (tgba_status is derived from them at the next sync).
enum : unsigned { kStNan = 1u, kStTableImag = 2u, kStTableSingular = 4u, kStTimeout = 8u, kStBadIndex = 16u,
                  kStEigen = 32u };

// Largest matrix (leading dimension, a multiple of 32) the native eigenvalue solver takes: its
// four length-ld vectors must fit in one CTA's shared memory.
constexpr int kMaxNativeLd = 6400;

// A contiguous run of states with the same quasiparticle number.
struct Group { int M; int64_t begin, end; };

struct Sector {
  int32_t m = 0;
  int64_t n_ns = 0, n_r = 0;
  int64_t ns_off = 0, r_off = 0;   // first state of the sector in the per-parity arrays
  int64_t x_off = 0;               // first element of the sector's X block ([n_ns][n_r])
  int64_t h_off = 0;               // first complex entry of the sector's H_eff
  int64_t ev_off = 0;              // first eigenvalue of the sector
  std::vector<Group> g_ns, g_r;
};

// Per-parity state tables, all sectors concatenated, in basis order.
struct StateTable {
  std::vector<double> E;
  std::vector<uint8_t> M;
  std::vector<int16_t> modes;      // [state][max_qp], ascending mode indices, -1 padded
};

// Work of the Pfaffian stage: a rectangle of pairs with uniform (M_a, M_b), laid out row-major
// (row = NS state, column = R state), cut into tiles of 32 consecutive pairs (one per warp).
struct Rect {
  int64_t out0;   // element index of the rectangle's first pair in the X cache
  int64_t ns0;    // global NS state index of the rectangle's first row
  int64_t r0;     // global R state index of the rectangle's first column
  int64_t tile0;  // index of the rectangle's first tile within its list
  int32_t ld;     // row stride of the sector's X block (n_r)
  int32_t w;      // rectangle width
  int32_t rows;   // rectangle height
  int32_t n;      // Pfaffian size M_a + M_b
  int32_t Ma;     // quasiparticles of the NS state
  int32_t pad;
};

// Rectangles of one size class: exact n for n <= 14 (register kernels), n <= 16/20/24/32 above.
struct RectList {
  int nmax = 0;
  std::vector<Rect> rects;        // sorted by n descending, tile0 prefix
  int64_t n_tiles = 0;
  Rect* d_rects = nullptr;
  int n_rects = 0;
};

// One kernel launch of the Pfaffian stage (kind 0: one exact register size, 1: queue over all
// register sizes, 2: shared-memory class).
struct PfLaunch { int kind, size, threads, grid, list; size_t smem; };
struct TuneEntry { int mode, threads; float ms; };

// Single-particle data of one parity at field h (Eq. 7, S3), host side.
struct Modes {
  int N = 0, parity = 0;
  double h = 0;
  std::vector<int> nlab;           // k = pi nlab / N, ascending
  std::vector<double> eps, theta, ex;
  double e_vac = 0, norm = 1;
};
Modes make_modes(int N, int parity, double h);

struct Basis;

// basis.cpp
tgba_status enumerate_basis(const tgba_model& model, const int32_t* sectors, int n_sectors,
                            const tgba_trunc& tr, Basis& b);
void build_rects(Basis& b);

struct Basis {
  int L = 0;
  double J = 1, h = 1;             // h = h_z / J
  int max_qp = 0;
  double e_cut = -1;
  int64_t cap = 0;
  double e_ns_vac = 0;             // NS vacuum energy (in units of J)
  std::vector<Sector> sectors;
  StateTable ns, r;
  int64_t n_elements = 0, n_heff = 0, n_states = 0;
  int max_n = 0;                   // largest M_a + M_b in the basis

  // device copies
  int device = 0;
  double* d_E_ns = nullptr; double* d_E_r = nullptr;
  uint8_t* d_M_ns = nullptr; uint8_t* d_M_r = nullptr;
  uint8_t* d_sel_ns = nullptr; uint8_t* d_sel_r = nullptr;   // [state][max_qp] table rows
  int16_t* d_modes_ns = nullptr; int16_t* d_modes_r = nullptr; // [state][max_qp] mode indices
  // mode data at h (host-computed, Eq. 7): theta of NS then R modes, and the labels n
  double* d_theta = nullptr;       // [2L]
  int* d_nlab = nullptr;           // [2L]
  double vac_norm = 1;             // n_NS n_R (Eq. S3)
  double norm_ns = 1, norm_r = 1;   // n_NS, n_R
  // contraction table
  double* d_table = nullptr;       // R, 2L x 2L row-major
  double* d_c0 = nullptr;          // C0 (re, im), then diagnostics: max |Im| residual, max |R|
  double c0_host[2] = {0, 0};
  double* d_work = nullptr;        // 4L x 4L complex scratch of the table build
  bool table_valid = false;
  // Pfaffian stage
  double* d_P = nullptr;           // X_ab = C0 (-i)^{(M_a+M_b)/2} P_ab, P real, [n_elements]
  bool x_valid = false;
  const void* x_screen = nullptr;
  double x_tau = 0;
  int64_t x_evaluated = 0, x_screened = 0;
  std::vector<RectList> rect_lists;    // one per size class (basis.cpp: tile_class)
  std::vector<Rect> reg_rects;         // all register-size rectangles, n descending, one tile prefix
  Rect* d_reg_rects = nullptr;
  int reg_rects_total = 0;
  int64_t reg_tiles_total = 0;
  int max_reg_n = 0;
  unsigned long long* d_counter = nullptr;   // work counter of the queue launch
  std::vector<PfLaunch> pf_plan;
  int tune_mode = 0, tune_threads = 128;
  bool tuned = false;
  std::vector<TuneEntry> tune_log;
  cudaGraph_t graph = nullptr;         // table + Pfaffian stage, captured once
  cudaGraphExec_t graph_exec = nullptr;
  bool c0_host_valid = false;
  int64_t graph_launches = 0;          // kernel launches inside the graph
  unsigned* d_status = nullptr;
  // measurement
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool ev_recorded = false;
  // native eigen-solver: events around its two kernels, work of the last batch
  cudaEvent_t eig_ev[3] = {nullptr, nullptr, nullptr};
  bool eig_ev_recorded = false;
  double tridiag_flops = 0;
  int64_t eig_matrices = 0;
  int eig_cluster = 0;
  std::atomic<int64_t> launches{0};
  int64_t upload_bytes = 0, pf_launches = 0;
  double pf_flops = 0;
  // eigen solver scratch
  void* solver = nullptr;          // cusolverDnHandle_t
  void* blas = nullptr;            // cublasHandle_t
  double* d_blas_ws = nullptr;     // its workspace (set explicitly, so captured calls allocate nothing)
  int emu_sms = 0;                 // SMs for the tensor-core FP64 products (emu_prepare)
  double* d_emu_part = nullptr;    // their partial tiles (emu_prepare)
  int quench_terms = 0;            // Chebyshev terms K of the last batched quench propagation
  double quench_flops = 0;         // its algorithmic FP64 flops (K sum 8 n_NS n_R)
  double quench_prep_ms = 0, quench_gram_ms = 0, quench_eval_ms = 0;   // its other stages
  cudaEvent_t q_ev[2] = {nullptr, nullptr};   // around its graph launch
  bool q_ev_recorded = false;
  double* d_eig_a = nullptr; double* d_eig_w = nullptr; double* d_eig_work = nullptr;
  double* d_scratch = nullptr; int64_t scratch_cap = 0;
  int* d_eig_info = nullptr;
  int64_t eig_a_cap = 0, eig_work_cap = 0;
};

// error helpers (api.cpp)
tgba_status fail(tgba_status st, const std::string& msg);
tgba_status cuda_fail(cudaError_t e, const char* what);

// table.cu
tgba_status build_table(Basis& b, cudaStream_t st);

// pfaffian.cu
tgba_status plan_pfaffians(Basis& b);
tgba_status autotune_pfaffians(Basis& b, cudaStream_t st);
tgba_status run_pfaffians(Basis& b, cudaStream_t st);
tgba_status run_pfaffian_pairs(Basis& b, int s, const int32_t* pairs, int64_t n, double* out, cudaStream_t st);
// direct.cu: X of explicit pairs by the paper-literal Pfaffian of size 2L + M_a + M_b
size_t x_direct_smem(int L, int max_qp, int jmid);
tgba_status x_direct(Basis& b, int s, const int32_t* pairs, int64_t n, double* out, cudaStream_t st);
// <phi_a| sigma^x_1 sigma^x_{jmid+1} |phi_b> for pairs of parity `parity` (jmid >= 0), or X (jmid < 0)
tgba_status direct_elements(Basis& b, int s, int parity, int jmid, const int32_t* pairs, int64_t n, double* out,
                            cudaStream_t st);
// reduced form of the same-parity elements: the contraction table of the string up to J
// (table.cu; S [2L + 2J]^2 complex, c0z one complex) and its Pfaffians (direct.cu)
tgba_status z_table(Basis& b, int parity, int J, double* S_dev, double* c0z_dev, cudaStream_t st);
size_t z_reduced_smem(int max_qp, int j);
tgba_status z_reduced_elements(Basis& b, int s, int parity, int j, int J, const double* S, const double* c0z,
                               const int32_t* pairs, int64_t n, double* out, cudaStream_t st);
// real P of every (NS state of sector s_ns, R state of sector s_r) pair, out [n_ns][n_r] row-major
tgba_status run_pfaffian_cross(Basis& b, int s_ns, int s_r, double* out, cudaStream_t st);

// assemble.cu
tgba_status assemble_heff(Basis& b, double h_x, double* heff, cudaStream_t st);
tgba_status export_x(Basis& b, int s, double* x, cudaStream_t st);
tgba_status build_real_heff(Basis& b, int s, double h_x, double* a, const int32_t* idx_ns, int64_t kn,
                            const int32_t* idx_r, int64_t kr, cudaStream_t st);

// eig.cu / quench.cu: library handles
void destroy_solver(void* h);
void destroy_blas(void* h);

// eig.cu
tgba_status eig_sym(Basis& b, int64_t n, double* a, double* w, bool vectors, cudaStream_t st);
// eigenvalues of every sector's real-gauge H_eff at each of n_hx fields, one batched solve;
// field h, sector s written at evals + h * n_states + ev_off.  method: 0 = native when every
// sector fits (n <= kMaxNativeLd), else the library; 1 = native; 2 = cuSOLVER XsyevBatched
tgba_status eig_all_sectors(Basis& b, const double* hx, int n_hx, double* evals, int method, cudaStream_t st);
// tridiag.cu: Householder tridiagonalisation by groups of CTAs + Sturm bisection.  check
// (optional): the group waits' poll limit and a CTA that leaves before its first barrier, to
// make the bounded waits run out (failure-detection checks)
struct WaitCheck {
  unsigned spin_limit;
  int withhold_matrix, withhold_rank;
};
tgba_status eig_all_sectors_native(Basis& b, const double* hx, int n_hx, double* evals, cudaStream_t st,
                                   const WaitCheck* check = nullptr);

// dsf.cu
tgba_status dsf(Basis& b, int s, double h_x, double w_min, double w_max, int n_w, double eta, float* S,
                double* evals, int n_ev, double* weights, double* dE, cudaStream_t st);

// S(k, w) at the momentum of sector s, ground state from the K = 0 sector s0
tgba_status dsf_k(Basis& b, int s, int s0, double h_x, double w_min, double w_max, int n_w, double eta, float* S,
                  double* evals, int n_ev, double* weights, double* dE, cudaStream_t st);

// quench.cu
// order 0: trunc = energy cutoffs above the NS vacuum (< 0: all); order 1: trunc = numbers of
// states chi, kept in order of |<phi|Phi0>|.  eps (optional, device, nv - 1): Eq. 11 between
// successive variants (they must be nested).
// j_max > 0 (eigen path): corr [nv][j_max][n_t] receives <sigma^x_1 sigma^x_{j+1}>(t) - <sigma^x>(t)^2
tgba_status quench(Basis& b, int s, double h0, const double* hx, const double* trunc, int nv, int order, double t_max,
                   int n_t, int method, double* mx, double* norm, double* eps, int64_t* chi, cudaStream_t st,
                   int j_max = 0, double* corr = nullptr);

// cheb.cu: batched Chebyshev propagation of quench variants whose kept sets are prefixes of one
// NS ranking and one R ranking.  Q: the X block of the union (col-major kr_max x kn_max), E:
// the union's energies (NS rows, then R rows), c: c~0 on the union (complex interleaved).
// Variant i writes mx[out][n_t].
struct ChebVariant {
  int out;
  int64_t kn, kr;
  double hx, norm2;
};
tgba_status quench_cheb_batch(Basis& b, const double* Q, int64_t kn_max, int64_t kr_max, const double* E,
                              const double* c, const std::vector<ChebVariant>& vars, double t_max, int n_t,
                              double* mx, cudaStream_t st);

// A pair kept by the screener: X element index and the global NS and R state indices.
struct PairEntry {
  int64_t out;
  int32_t a, b;
};
// screen_tc.cu: tensor-core scoring of the pairs of `rects` (see the file); pred (optional) gets
// y at (element index - pred_base); counts/list_off/lists (optional) receive the kept pairs per
// size n / 2.  Apart/Bpart: layer-1 partials of every NS / R state of the basis (global index).
tgba_status score_rects_tc(Basis& b, const std::vector<Rect>& rects, const float* Apart, const float* Bpart,
                           const __nv_bfloat16* W2b, const float* b2, const float* w3, const float* b3, float shift,
                           float half_log_l, float* pred, int64_t pred_base, unsigned* counts,
                           const int64_t* list_off, PairEntry* lists, cudaStream_t st);
// pfaffian.cu: Pfaffians of the kept pairs (sizes n <= 14, lists per n / 2), and the launches of
// the shared-memory size classes (n >= 16) without screening
tgba_status run_pfaffian_lists(Basis& b, const unsigned* counts, const int64_t* list_off, const PairEntry* lists,
                               cudaStream_t st);
tgba_status run_pfaffians_smem_classes(Basis& b, cudaStream_t st);

// dgemm_tc.cu: FP64 products on the tensor cores (BF16 slices, exact FP32 chunk sums, 48-bit
// running sums).  An operand (rows x K) is sliced by emu_slice into tile images of 128 rows (A
// and B); emu_gemm computes C = A B^T over a list of output tiles (row block, column block,
// columns used n_eff (a multiple of 16, <= 128), K blocks nkb, and per 16-column group the K
// blocks gkb that its columns reach (0: all nkb); B must be zero beyond them).  The chunks of
// all tiles are split evenly over the SMs; emu_number_tiles numbers them (c0) and zeroes the
// arrival counters, which the kernel leaves at zero again.
struct EmuTile {
  int32_t rb, cb, n_eff, nkb;
  int64_t c0;                 // first chunk of the tile in the list's order
  int32_t arrivals[8];        // CTAs done with each epilogue warp's block of a split tile
  int16_t gkb[8];             // K blocks per 16-column group
};
size_t emu_operand_elems(int rows, int K, int tile_rows);
int emu_tile_rows_a();
int emu_tile_rows_b();
int emu_k_block();
tgba_status emu_slice(Basis& b, const double* src, int64_t row_stride, int64_t k_stride, int k_split, int64_t k_jump,
                      const double* w, double w_shift, int rows, int K, int tile_rows, __nv_bfloat16* out, int* e,
                      cudaStream_t st);
tgba_status emu_prepare(Basis& b);
size_t emu_part_bytes(int sms);
int64_t emu_number_tiles(std::vector<EmuTile>& tiles);     // total chunks; -1 for an invalid tile
tgba_status emu_gemm(Basis& b, const __nv_bfloat16* A, const int* ea, int M, int Ka, const __nv_bfloat16* B,
                     const int* eb, int N, int Kb, EmuTile* d_tiles, int n_tiles, int64_t n_chunks, double* C,
                     int64_t ldc, cudaStream_t st, int n_slices = 6);   // 2: only the two leading digits (~2^-16)

// screen.cu
struct Screen;
tgba_status screen_create(int H, const float* params, uint64_t seed, Screen** out);
void screen_free(Screen* s);
int64_t screen_nparams(const Screen* s);
tgba_status screen_params(Screen& s, float* host);
tgba_status screen_grad(Screen& s, const float* x, const float* t, int64_t B, float* grad, double* loss, cudaStream_t st);
tgba_status screen_train(Basis** sets, int n_sets, int64_t n_samples, uint64_t seed, int H, int epochs, Screen** out,
                         double* stats, cudaStream_t st);
tgba_status screen_score(Screen& s, Basis& b, int sidx, float* pred, cudaStream_t st);
tgba_status screen_pfaffians(Screen& s, Basis& b, double tau, double hx, int64_t* kept, cudaStream_t st);

// status word
tgba_status check_status(Basis& b, cudaStream_t st);

// device scratch owned by the handle (grown on demand)
tgba_status scratch(Basis& b, int64_t doubles, double** out);

// peak.cu
tgba_status fp64_peak(int reps, double* gflops);

}  // namespace tgba

#define TGBA_CUDA(call)                                            \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::tgba::cuda_fail(e_, #call);    \
  } while (0)
