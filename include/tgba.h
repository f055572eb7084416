/*
 * tgba.h - C ABI of the GB300 TGBA library (libtgba.so).
 *
 * The Truncated Gaussian Basis Approach (arXiv:2410.04204) for the Ising chain
 *     H = -sum sx_j sx_{j+1} - h_z sum sz_j - h_x sum sx_j      (Eq. 3, periodic, L even)
 * builds, per momentum sector, the effective Hamiltonian
 *     H_ab = E^(0)_a delta_ab + <phi_a|V|phi_b>                  (Eq. 2)
 * over retained eigenstates phi of the free part H0 (fermionic Gaussian states, Eq. 6-7),
 * with <phi_a|V|phi_b> = -L h_x <phi_a|c_1 + c_1^dag|phi_b> (Eq. S4) evaluated as Pfaffians
 * (Eq. S1-S2), diagonalises it (Eq. 1), and evaluates the dynamic structure factor (Eq. 9)
 * and quench dynamics (Eq. 10).
 *
 * Conventions shared by every call
 *  - Errors: every call returns a tgba_status; nothing throws across the ABI.  Argument errors
 *    are detected on the host before any launch.  tgba_last_error() returns a thread-local
 *    message for the last failing call on this thread.  There is no CPU fallback: without a
 *    usable CUDA device, calls that compute return TGBA_ECUDA.
 *  - Ownership: handles (tgba_basis, tgba_screen) are created and freed by the library and
 *    own the device memory they need.  Output buffers are allocated by the caller; "_dev"
 *    arguments are device pointers, "_host" arguments host pointers.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *    device work of a call is ordered on that stream; calls return once the work is enqueued
 *    unless stated otherwise.  Device-side numeric faults (a NaN pivot, a non-real contraction
 *    table) are reported through a status word that the next synchronising call reads.
 *  - Complex numbers are interleaved (re, im) pairs of doubles (complex128).
 *  - Basis order inside a sector: the NS states (fermion parity Q = +1) first, then the R states
 *    (Q = -1); within a parity by quasiparticle number M, then energy, then mode indices.
 *  - Modes: mode index i of parity P is momentum k = pi n / L with n = -(L-1) + 2i (NS) or
 *    n = -(L-2) + 2i (R; i = L-1 is k = pi), i.e. modes in ascending k.
 */
#ifndef TGBA_H
#define TGBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TGBA_OK = 0,
  TGBA_EINVAL = 1,     /* bad argument (checked on the host, nothing launched) */
  TGBA_ENOMEM = 2,     /* device or host allocation failed */
  TGBA_ECUDA = 3,      /* CUDA / cuSOLVER error, or no usable device */
  TGBA_ENUMERIC = 4,   /* NaN/Inf in a Pfaffian, singular vacuum block, non-real table */
  TGBA_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  TGBA_ELIMIT = 6      /* a size limit of the library was exceeded */
} tgba_status;

/* Model (Eq. 3).  L even, 4 <= L <= 120; J > 0 (energies scale as H(J,h,hx) = J H(1,h/J,hx/J)).
   h_z > 0 is the transverse field.  h_x is not used by tgba_build_basis (V enters later). */
typedef struct { int32_t L; double J; double h_z; double h_x; } tgba_model;

/* Truncation (Method section; Appendix B).  Keep states with M <= max_qp quasiparticles
   (0 <= max_qp <= 16, even M only) and, if e_cut >= 0, energy E - E_NS,vacuum <= e_cut (+1e-9);
   then, if max_per_parity > 0, the max_per_parity lowest in (E, M, modes) of each parity. */
typedef struct { int32_t max_qp; double e_cut; int64_t max_per_parity; } tgba_trunc;

typedef struct tgba_basis_s* tgba_basis;     /* opaque, library-owned */
typedef struct tgba_screen_s* tgba_screen;   /* opaque, library-owned */

/* Thread-local description of the last error on this thread ("" if none). */
const char* tgba_last_error(void);

/* Number of CUDA devices the library can use (0 if none); never fails. */
int32_t tgba_device_count(void);

/* ---------------------------------------------------------------- basis (Eq. 6-7, Method)
 * Enumerate, per requested momentum sector K = 2 pi m / L, the H0 eigenstates
 * d^dag_{k1}...d^dag_{kM}|0>_{NS/R} (M even, sum k = K mod 2 pi), truncate them, and upload the
 * state tables to the current device.  sectors_m: n_sectors distinct values in [0, L).
 * Host work plus synchronous uploads; on success *out owns device memory until
 * tgba_basis_free.  TGBA_ELIMIT if a sector would exceed 2^31 elements. */
tgba_status tgba_build_basis(const tgba_model* model, const int32_t* sectors_m, int32_t n_sectors,
                             const tgba_trunc* trunc, tgba_basis* out);

/* Sizes and (optionally) state data of sector index s (0 <= s < n_sectors).
   n_ns, n_r: number of NS and R states.  Optional host outputs (NULL to skip), each sized for
   n_ns + n_r states in basis order: E0 (energies E^(0)), parity (0 = NS, 1 = R), nqp (M) and
   modes ([state][max_qp] ascending mode indices, -1 padded). */
tgba_status tgba_basis_info(tgba_basis b, int32_t s, int64_t* n_ns, int64_t* n_r, double* E0_host,
                            uint8_t* parity_host, uint8_t* nqp_host, int16_t* modes_host);

/* Totals: number of sectors, sum over sectors of n_ns * n_r (the Pfaffian elements) and of
   (n_ns + n_r)^2 (the H_eff entries, i.e. the complex128 count tgba_assemble_heff writes). */
tgba_status tgba_basis_totals(tgba_basis b, int32_t* n_sectors, int64_t* n_elements, int64_t* n_heff);

tgba_status tgba_basis_free(tgba_basis b);

/* ---------------------------------------------------------------- Pfaffian stage (App. A)
 * Computes, for every sector, X_ab = <phi_a^NS| c_1 + c_1^dag |phi_b^R> (Eq. S4) for all NS x R
 * pairs and keeps them in the basis handle (device memory owned by the library), where
 * tgba_assemble_heff, tgba_dsf and tgba_quench reuse them for any h_x.  Steps: the
 * contraction table of the Bogoliubov operators (the Schur complement of Eq. S2's matrix on
 * the vacuum operators) and then one small real Pfaffian per element, of size M_a + M_b,
 * batched over all sectors and sizes.  screen: NULL for the exact assembly, or a trained pair
 * screener; pairs it predicts with |V_ab| = L h_x |X_ab| < screen_tau (at screen_hx) are set to
 * 0 without a Pfaffian.  Asynchronous on `stream`. */
tgba_status tgba_compute_x(tgba_basis b, tgba_screen screen, double screen_tau, double screen_hx, void* stream);

/* Number of pairs the last tgba_compute_x evaluated by Pfaffian (after screening); blocks on
   the stream of that call. */
tgba_status tgba_x_stats(tgba_basis b, int64_t* n_evaluated, int64_t* n_screened);

/* Copy sector s's X block, complex128 [n_ns][n_r] row-major in basis order, to x_dev. */
tgba_status tgba_x_export(tgba_basis b, int32_t s, double* x_dev, void* stream);

/* X for an explicit list of pairs of sector s: pairs_dev int32 [n][2] = (NS index, R index)
   in basis order; out_dev complex128 [n].  Uses the contraction table (computing it if needed).  Indices outside the sector give
   TGBA_EINVAL (NaN is written for them); blocks on `stream`. */
tgba_status tgba_x_pairs(tgba_basis b, int32_t s, const int32_t* pairs_dev, int64_t n_pairs,
                         double* out_dev, void* stream);

/* X for explicit pairs, as tgba_x_pairs, but evaluated the paper-literal way (Appendix A,
   Eq. S1-S2): the vacuum expectation of the whole string of 2L + M_a + M_b Bogoliubov operators
   (both vacua, the excitations and sigma^x_1, expanded on the lattice sites), one complex
   Pfaffian of that size per element, a warp each.  O((2L)^3) per element instead of the
   reduced form's O((M_a + M_b)^3): a GPU cross-check of tgba_x_pairs and an FP64-dense workload.
   Needs one warp's dense 2L + 2 max_qp string in shared memory: TGBA_EINVAL when it does not
   fit (L = 60 with max_qp = 16 fits).  Pair and output layout, index checks as tgba_x_pairs;
   blocks on `stream`. */
tgba_status tgba_x_direct(tgba_basis b, int32_t s, const int32_t* pairs_dev, int64_t n_pairs, double* out_dev,
                          void* stream);

/* Elements Z_ab = <phi_a| sigma^x_1 sigma^x_{j+1} |phi_b> between two states of parity `parity`
   (0 = NS, 1 = R) of sector s, 0 <= j < L (j = 0: the overlap <phi_a|phi_b>).  After the
   Jordan-Wigner map the operator is the string B_1 A_2 B_2 ... B_j A_{j+1} of 2j Majoranas
   (A_l = c_l^dag + c_l, B_l = c_l^dag - c_l) between vacua of one parity, the structure of
   Eq. S1-S2 with the string in place of sigma^x_1.  Reduced form: the two vacua are contracted
   once (a Schur complement whose pivot block has the vacuum norm as Pfaffian), leaving a table
   over the excitation operators and the string, and each element is a Pfaffian of size
   M_a + 2j + M_b (shared memory bounds max_qp and j: TGBA_EINVAL when it does not fit).
   pairs_dev: int32 [n_pairs][2] state indices within the sector's states of that parity;
   out_dev: complex (re, im) [n_pairs]; TGBA_EINVAL on an out-of-range index (output NaN).
   Blocks on `stream`. */
tgba_status tgba_z_elements(tgba_basis b, int32_t s, int32_t parity, int32_t j, const int32_t* pairs_dev,
                            int64_t n_pairs, double* out_dev, void* stream);

/* Contraction table and vacuum element: c0_host (complex, 2 doubles) receives
   C0 = <0_NS|c_1 + c_1^dag|0_R>; table_dev (optional, 2L x 2L doubles row-major) receives the
   real table R.  Blocks on `stream`. */
tgba_status tgba_table(tgba_basis b, double* c0_host, double* table_dev, void* stream);

/* ---------------------------------------------------------------- H_eff (Eq. 2, S4)
 * Writes, for every sector in order, H = diag(E^(0)) - L h_x [[0, X], [X^H, 0]] as a dense
 * complex128 (n x n, n = n_ns + n_r) column-major matrix; the sectors follow each other in
 * heff_dev (total size from tgba_basis_totals).  Runs tgba_compute_x(b, screen, ...) first if
 * the handle holds no X for that screen.  Asynchronous on `stream`. */
tgba_status tgba_assemble_heff(tgba_basis b, double h_x, tgba_screen screen, double screen_tau,
                               double* heff_dev, void* stream);

/* ---------------------------------------------------------------- diagonalisation (Eq. 1)
 * All eigenvalues, ascending, of the H_eff that tgba_assemble_heff writes, for each of the n_hx
 * longitudinal fields h_x[i], computed from the handle's X.  evals_dev: double
 * [n_hx][n_states] (n_states = sum over sectors of n_ns + n_r); field i, sector s starts at
 * i * n_states + (sum of the sizes of sectors before s).  The sector matrices are real
 * symmetric after a diagonal change of phase of the basis states, so every (field, sector)
 * matrix goes into one batched FP64 real symmetric solve.  method (tgba_eigvals_ex):
 *   0  automatic: 1 when every sector has at most 6400 states (rounded up to a multiple of
 *      32), else 2;
 *   1  native: Householder tridiagonalisation, a group of CTAs per matrix (one cooperative
 *      launch, SMs shared out by work), then bisection on Sturm counts, the first steps in
 *      single precision within a proven bracket and the last in FP64 to 4 eps ||T||
 *      (TGBA_EINVAL if a sector is too large; TGBA_ETIMEOUT if a bounded device wait of the
 *      tridiagonalisation gave up);
 *   2  cuSOLVER XsyevBatched, each matrix padded to the largest sector size with decoupled
 *      diagonal entries above its Gershgorin bound.
 * A non-finite matrix entry gives TGBA_ENUMERIC.  tgba_eigvals is method 0.  Blocks on `stream`. */
tgba_status tgba_eigvals(tgba_basis b, const double* h_x, int32_t n_hx, double* evals_dev, void* stream);
tgba_status tgba_eigvals_ex(tgba_basis b, const double* h_x, int32_t n_hx, int32_t method, double* evals_dev,
                            void* stream);

/* Failure-detection check of the bounded waits of the native solver (method 1); not in the
   paper.  The CTAs of a group that works on one matrix meet at barriers in global memory whose
   waits are bounded: after spin_limit polls (about 100 ns each; the normal limit is 2^24) a
   wait gives up, sets a status bit and the group leaves the matrix, so a lost CTA can never
   hang the GPU.  This call runs tgba_eigvals_ex(method 1) with the given poll limit and, if
   withhold_matrix >= 0, with the CTA of rank withhold_rank in the group of the
   withhold_matrix-th (field, sector) matrix (fields outer, sectors inner, empty sectors
   skipped) leaving before its first barrier, so that its group waits for an arrival that never
   comes.  The result is then TGBA_ETIMEOUT (the status word is cleared and the handle stays
   usable; the eigenvalues of that matrix are meaningless).  TGBA_EINVAL if that CTA's group has
   fewer than two CTAs (nothing would wait) or the rank is outside it.  Blocks on `stream`. */
tgba_status tgba_eigvals_wait_check(tgba_basis b, const double* h_x, int32_t n_hx, uint32_t spin_limit,
                                    int32_t withhold_matrix, int32_t withhold_rank, double* evals_dev, void* stream);

/* ---------------------------------------------------------------- S(k=0, w) (Eq. 8-9)
 * Dynamic structure factor of sector index s (which must be the k = 0 sector, m = 0):
 * S(w_i) = 2 pi sum_a w_a L_eta(w_i - (E_a - E_0)), w_a = L |<psi_0|sigma^x_1|psi_a>|^2,
 * L_eta(x) = (eta/pi)/(x^2 + eta^2), w_i = w_min + i (w_max - w_min)/(n_w - 1).
 * Weights in FP64; the Lorentzian sum in FP32 with FP32 accumulation.  S_dev: float [n_w].
 * Optional: evals_dev (double, first n_ev eigenvalues), weights_dev (double [n], w_a) and
 * dE_dev (double [n], E_a - E_0).  Blocks on `stream`. */
tgba_status tgba_dsf(tgba_basis b, int32_t s, double h_x, double w_min, double w_max, int32_t n_w, double eta,
                     float* S_dev, double* evals_dev, int32_t n_ev, double* weights_dev, double* dE_dev,
                     void* stream);

/* S(k, w) at the momentum k = 2 pi m / L of sector s (Eq. 8-9 with the matrix element that follows
   them, <psi_a^k|sigma^x_k|psi_0> = sqrt(L) e^{-ik} <psi_a^k|sigma^x_1|psi_0>): S(w_i) =
   2 pi sum_a w_a L_eta(w_i - (E_a - E_0)) over the eigenstates a of sector s, w_a =
   L |<psi_a|sigma^x_1|psi_0>|^2, with psi_0, E_0 the ground state of sector s0, which must be
   the k = 0 sector of the basis.  sigma^x_1 connects NS states of one sector with R states of the
   other, and these cross-sector elements are computed here, as Pfaffians of the same contraction
   table.  Grid, eta, outputs and their layout as in tgba_dsf (evals/weights/dE are those of sector
   s; dE relative to E_0).  s = s0 gives tgba_dsf's result.  Needs tgba_compute_x first; blocks on
   `stream`. */
tgba_status tgba_dsf_k(tgba_basis b, int32_t s, int32_t s0, double h_x, double w_min, double w_max, int32_t n_w,
                       double eta, float* S_dev, double* evals_dev, int32_t n_ev, double* weights_dev, double* dE_dev,
                       void* stream);

/* ---------------------------------------------------------------- quench (Eq. 10)
 * <sigma^x>(t) after the quench from Phi0 = (|0_NS(h_z0)> + s|0_R(h_z0)>)/sqrt 2 (ground states
 * of the h_x = 0 chain at h_z0, s making <sigma^x>(0) > 0) to the basis' model with
 * longitudinal field hx_variants[v].  Sector index s must be k = 0.  Variant v keeps the states
 * of the basis with E - E_NS,vacuum <= ecut_variants[v] (+1e-9; a negative value keeps all), so
 * variants with growing cutoffs are nested truncations (Method section, Fig. 2: several chi).
 * B(t) = M^T e^{-iEt} M^* c0 with c0 = <phi|Phi0> (Eq. S6), <sigma^x>(t) = B^H X B / ||c0||^2
 * on t_i = i t_max/(n_t - 1).  method: 1 diagonalises H_eff (FP64 syevd) and forms B(t) from its
 * eigenpairs, as Eq. 10 writes it; 2 expands e^{-iH t} c0 = B(t) in Chebyshev polynomials of the
 * rescaled H_eff with Bessel coefficients (Jacobi-Anger), truncated where J_k(R t_max) < 1e-16,
 * which needs only products with H_eff and lifts the cubic cost of the diagonalisation; 0 picks 1
 * up to 4096 retained states and 2 above.  mx_dev: double [n_variants][n_t]; norm_dev (optional):
 * double [n_variants], ||c0||^2 of each variant; chi_host (optional): int64 [n_variants], the
 * retained basis size of each variant.  Blocks on `stream`. */
tgba_status tgba_quench(tgba_basis b, int32_t s, double h_z0, const double* hx_variants,
                        const double* ecut_variants, int32_t n_variants, double t_max, int32_t n_t, int32_t method,
                        double* mx_dev, double* norm_dev, int64_t* chi_host, void* stream);

/* The quench with the paper's choice of truncated subspace (the Quench section): the states of
   the k = 0 sector s are ranked by bare energy (order 0) or by |<phi|Phi0>|, largest first, ties
   by energy (order 1), and variant v keeps, in this ranking, the states with
   E - E_NS,vac <= trunc_variants[v] (order 0; a negative value keeps all) or the first
   trunc_variants[v] states (order 1; a whole number >= 1).  mx_dev, norm_dev, chi_host as in
   tgba_quench.  eps_dev (optional, device, n_variants - 1 doubles): the convergence metric of
   Eq. 11, eps(chi_{v+1}, chi_v) = max over the time grid of || Psi^{chi_v}(t) -
   Psi^{chi_{v+1}}(t) ||; it needs nested variants (non-decreasing trunc_variants, else
   TGBA_EINVAL) and the eigendecomposition path (method 1, or method 0 with at most 4096 states
   per variant).  tgba_quench is order 0 without eps.  Blocks on `stream`. */
tgba_status tgba_quench_ordered(tgba_basis b, int32_t s, double h_z0, const double* hx_variants,
                                const double* trunc_variants, int32_t n_variants, int32_t order, double t_max,
                                int32_t n_t, int32_t method, double* mx_dev, double* norm_dev, double* eps_dev,
                                int64_t* chi_host, void* stream);

/* Equal-time connected correlators after the quench (the correlation-function passage of the
   appendix): C_j(t) = <sigma^x_1(t) sigma^x_{j+1}(t)> - <sigma^x(t)>^2 for j = 1..j_max, in the
   truncated subspace of one variant (h_x, trunc, order as one variant of tgba_quench_ordered),
   with expectation values in the normalised state (the k = 0 state is translation invariant,
   so <sigma^x_{j+1}> = <sigma^x_1>).  After the Jordan-Wigner map sigma^x_1 sigma^x_{j+1} is a
   string of 2j Majorana operators; its NS-NS and R-R elements are those of tgba_z_elements
   (reduced-form Pfaffians of size M_a + M_b + 2j, so max_qp and j_max are bounded by shared
   memory: TGBA_EINVAL when they do not fit; 1 <= j_max < L).  Eigendecomposition path.
   mx_dev: double [n_t]; corr_dev: double [j_max][n_t]; norm_dev (optional): ||c0||^2;
   chi_host (optional): the kept basis size.  Blocks on `stream`. */
tgba_status tgba_quench_correlators(tgba_basis b, int32_t s, double h_z0, double h_x, double trunc, int32_t order,
                                   double t_max, int32_t n_t, int32_t j_max, double* mx_dev, double* corr_dev,
                                   double* norm_dev, int64_t* chi_host, void* stream);

/* ---------------------------------------------------------------- learned pair screener
 * Not in the paper (the paper has no counterpart): a 3-layer MLP (width 256, ReLU, FP32
 * parameters) that predicts log10|X_ab| from the two quasiparticle momentum sets, trained on
 * exact elements of the Pfaffian path, and used by tgba_compute_x to skip the Pfaffians of pairs
 * it predicts below the threshold.  Features (D = 20): k/pi of the NS state's modes (ascending,
 * zero padded to 8), k/pi of the R state's modes, M_a/8, M_b/8, 24/L, 1.  Target:
 * log10|X| + (M_a+M_b)/2 log10(L/24), clipped at -30.  Parameters, flat FP32: W1 [256][20],
 * b1 [256], W2 [256][256], b2 [256], w3 [256], b3 [1].  A pair is skipped when
 * predicted log10|V| = y - (M_a+M_b)/2 log10(L/24) + log10(L |h_x|) < log10(tau) - margin, with
 * margin = 3 x the validation RMSE of training (always kept: states with more than 8
 * quasiparticles).  Layer 2 of the inference runs on the tensor cores in BF16. */

/* A screener with the given parameters (params_host: n floats, see above) or, if params_host is
   NULL, He-normal weights drawn from `seed`.  width must be 256. */
tgba_status tgba_screen_create(int32_t width, const float* params_host, uint64_t seed, tgba_screen* out);
tgba_status tgba_screen_nparams(tgba_screen s, int64_t* n);
tgba_status tgba_screen_params(tgba_screen s, float* params_host);
/* Forward and back-propagation of one batch (no update): x_dev float [B][20], t_dev float [B];
   grad_dev float [nparams] receives d(mean (y - t)^2)/d params, loss_host the loss. */
tgba_status tgba_screen_grad(tgba_screen s, const float* x_dev, const float* t_dev, int64_t B, float* grad_dev,
                             double* loss_host, void* stream);
/* Train a new screener on n_samples pairs drawn uniformly (SplitMix64 from `seed`) from all
   NS x R pairs of the given bases, labelled by their exact X: Adam, batches of 4096, `epochs`
   passes, the last 5 % held out.  stats_host (optional, 4 doubles): train RMSE, validation RMSE,
   margin, seconds.  Blocks on `stream`. */
tgba_status tgba_screen_train(const tgba_basis* sets, int32_t n_sets, int64_t n_samples, uint64_t seed,
                              int32_t width, int32_t epochs, tgba_screen* out, double* stats_host, void* stream);
/* Predicted y (see above) of every pair of sector s: pred_dev float [n_ns][n_r]. */
tgba_status tgba_screen_predict(tgba_screen s, tgba_basis b, int32_t sector, float* pred_dev, void* stream);
tgba_status tgba_screen_free(tgba_screen s);

/* ---------------------------------------------------------------- allocation-free table
 * The paper has no counterpart: this is a service entry point of the library.  It computes the
 * same contraction table and vacuum element as tgba_table, but for callers that cannot let the
 * library allocate device memory, for example a process whose device memory belongs to a
 * fixed-size pool that refuses allocations made behind its back, or a latency-critical loop
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.  Nothing is allocated:
 * the work matrix (4L x 4L complex) and the per-call inputs live in statically sized device
 * arrays of the library (about 1 MiB, held on every GPU that loads the library until the
 * process exits), so L is limited to 64 (TGBA_ELIMIT beyond).  The first call on a device, and
 * the first after a cudaDeviceReset, looks up the device addresses of those arrays
 * (cudaGetSymbolAddress, which may load the library's device code); make that call before any
 * stream capture begins.  Every call waits for its work to finish: it reads a status word back
 * to the host.  All calls share the arrays, which keep the last call's contents: calls that
 * overlap on the GPU, from any thread or stream, race and must be serialised by the caller.
 * table_dev: caller-owned double [2L][2L] (row-major, the real table R of tgba_table); c0_dev:
 * caller-owned double [2] receiving C0 = <0_NS|c_1 + c_1^dag|0_R>.  Blocks on `stream`. */
tgba_status tgba_table_noalloc(int32_t L, double J, double h_z, double* table_dev, double* c0_dev, void* stream);

/* ---------------------------------------------------------------- measurement
 * Profile of a basis handle.  table_ms / pfaffian_ms: device time of the contraction table and
 * of the Pfaffian kernels of the last tgba_compute_x, from CUDA events recorded on its stream
 * (blocks until they complete).  pfaffian_flops: algorithmic FP64 flops of one Pfaffian stage,
 * sum over elements of F(n) = sum_{m = n-2, n-4, ..., 2} [2 m (m-1) + m] (the real-arithmetic
 * Parlett-Reid count: two FMAs per updated entry, one multiply per Gauss-vector entry).
 * pfaffian_launches: kernel launches of one Pfaffian stage.  kernel_launches: all kernel
 * launches this handle has made (this library's kernels only, not cuSOLVER/cuBLAS).
 * upload_bytes: host-to-device bytes of tgba_build_basis.  tune_mode / tune_threads: the launch
 * shape the autotuner chose for the register-resident sizes (0: one launch per size, 1: one
 * persistent queue launch, 3: the queue with a register cap for occupancy; threads per block),
 * tune_ms: its measured stage time (ms) for each candidate in the order {0,64}, {0,128},
 * {0,256}, {1,64}, {1,128}, {1,256}, {3,128} (0 where not measured).
 * tridiag_ms / bisect_ms: device time of the tridiagonalisation and of the bisection kernel of
 * the last native tgba_eigvals (0 if none ran); tridiag_flops: its algorithmic FP64 flops,
 * sum over matrices of sum_{m=1}^{n-1} 4 m (m + 1) (two FMAs of the rank-2 update and two of
 * the symmetric product per element of the trailing lower triangle, ~4n^3/3); eig_matrices:
 * matrices in that batch; eig_cluster: CTAs per matrix.
 * quench_ms: device time of the last batched Chebyshev propagation of tgba_quench (the graph of
 * its K steps over all variants); quench_terms: K; quench_flops: its algorithmic FP64 flops,
 * K sum over variants of 8 n_NS n_R (two real vectors, both off-diagonal blocks, one FMA per
 * entry); quench_prep_ms, quench_gram_ms, quench_eval_ms: host-clock times of its other
 * stages (the slicing of X and the Lanczos bounds; the moments; the Bessel sums over the time
 * grid). */
typedef struct {
  double table_ms, pfaffian_ms, pfaffian_flops;
  int64_t pfaffian_launches, kernel_launches, upload_bytes, evaluated;
  int32_t tune_mode, tune_threads;
  double tune_ms[8];
  double tridiag_ms, bisect_ms, tridiag_flops;
  int64_t eig_matrices;
  int32_t eig_cluster, pad_;
  double quench_ms, quench_flops;
  int64_t quench_terms;
  double quench_prep_ms, quench_gram_ms, quench_eval_ms;
} tgba_prof;
tgba_status tgba_profile(tgba_basis b, tgba_prof* out);

/* ---------------------------------------------------------------- FP64 products on the tensor cores
 * Not in the paper: the FP64 matrix products of the batched quench propagation run through
 * this routine, exposed for direct use and testing.  C = A B^T with A [M][K] (row i at A + i lda,
 * K contiguous), B [N][K] (row j at B + j ldb), C column-major M x N (entry (i, j) at
 * C + i + j ldc); all device pointers, FP64.  Each operand row is scaled by a power of two and cut
 * into six signed 8-bit digits held exactly in BF16; the tensor cores (tcgen05 MMAs, FP32
 * accumulation in tensor memory) sum the digit products, exactly for the three leading digit
 * diagonals over chunks of 256 K values, and the chunks are added into a 48-bit running sum
 * (a pair of FP32 numbers).  The error is a few 1e-13 of sum_k |A_ik B_jk| (below 1e-12).  M, N, K >= 1
 * (TGBA_EINVAL otherwise); the slice buffers (12 bytes per input element) are allocated for the
 * call (TGBA_ENOMEM).  Blocks on `stream`. */
tgba_status tgba_dgemm_tc(int32_t M, int32_t N, int32_t K, const double* A, int64_t lda, const double* B, int64_t ldb,
                          double* C, int64_t ldc, void* stream);

/* ---------------------------------------------------------------- measurement helper
 * Achieved FP64 rate of a DFMA-chain kernel on the current device (GFLOP/s, best of `reps`),
 * the denominator for FP64 roofline fractions. */
tgba_status tgba_fp64_peak(int32_t reps, double* gflops);

#ifdef __cplusplus
}
#endif
#endif /* TGBA_H */
