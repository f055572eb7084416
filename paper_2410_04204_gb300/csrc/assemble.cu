// Effective Hamiltonian (row a6; Eq. 2 and Eq. S4):
//   H = diag(E^(0)) - L h_x [[0, X], [X^H, 0]],  X_ab = C0 (-i)^{(M_a+M_b)/2} P_ab.
// With the diagonal unitary G = diag(g), g_a = (-i)^{M_a/2} on NS states and
// g_b = i^{M_b/2} e^{-i arg C0} on R states, G^H H G is real symmetric with off-diagonal block
// -L h_x |C0| P; the eigen solver and the spectral sums work in that gauge (eigenvalues and
// |<psi|sigma|psi'>| are unchanged).
#include "tgba_internal.h"

namespace tgba {
namespace {

// X_ab from P_ab
__device__ __forceinline__ double2 xval(const double* c0, double p, int n) {
  const double re = c0[0] * p, im = c0[1] * p;
  switch ((n >> 1) & 3) {
    case 0: return make_double2(re, im);
    case 1: return make_double2(im, -re);
    case 2: return make_double2(-re, -im);
    default: return make_double2(-im, re);
  }
}

// Column-major complex H of one sector, one thread per entry in 32 x 32 blocks of entries.  The
// writes are coalesced; in the NS-row/R-column block the reads of P stride by n_r.
__global__ void heff_kernel(int64_t n_ns, int64_t n_r, const double* __restrict__ E_ns, const double* __restrict__ E_r,
                            const uint8_t* __restrict__ M_ns, const uint8_t* __restrict__ M_r,
                            const double* __restrict__ P, const double* __restrict__ c0, double scale,
                            double2* __restrict__ H) {
  const int64_t n = n_ns + n_r;
  const int64_t col0 = (int64_t)blockIdx.y * 32, row0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t col = col0 + yy, row = row0 + tx;
    if (col >= n || row >= n) continue;
    double2 v = make_double2(0.0, 0.0);
    if (row == col) {
      v.x = row < n_ns ? E_ns[row] : E_r[row - n_ns];
    } else if (col < n_ns && row >= n_ns) {            // R row, NS column: -L h_x conj(X_{col, row-n_ns})
      const int64_t a = col, b = row - n_ns;
      double2 x = xval(c0, P[a * n_r + b], M_ns[a] + M_r[b]);
      v = make_double2(scale * x.x, -scale * x.y);
    } else if (col >= n_ns && row < n_ns) {            // NS row, R column: -L h_x X_{row, col-n_ns}
      const int64_t a = row, b = col - n_ns;
      double2 x = xval(c0, P[a * n_r + b], M_ns[a] + M_r[b]);
      v = make_double2(scale * x.x, scale * x.y);
    }
    H[col * n + row] = v;
  }
}

// Real-gauge H~ (column-major, n_k x n_k) of a subset of a sector's states.
__global__ void heff_real_kernel(int64_t kn, int64_t kr, const int32_t* __restrict__ idx_ns,
                                 const int32_t* __restrict__ idx_r, int64_t n_r, const double* __restrict__ E_ns,
                                 const double* __restrict__ E_r, const double* __restrict__ P,
                                 const double* __restrict__ c0, double scale, double* __restrict__ A) {
  const int64_t n = kn + kr;
  const double c = scale * sqrt(c0[0] * c0[0] + c0[1] * c0[1]);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = idx / n, row = idx - col * n;
    double v = 0.0;
    if (row == col) {
      v = row < kn ? E_ns[idx_ns ? idx_ns[row] : row] : E_r[idx_r ? idx_r[row - kn] : row - kn];
    } else if (row < kn && col >= kn) {
      const int64_t a = idx_ns ? idx_ns[row] : row, b = idx_r ? idx_r[col - kn] : col - kn;
      v = c * P[a * n_r + b];
    } else if (row >= kn && col < kn) {
      const int64_t a = idx_ns ? idx_ns[col] : col, b = idx_r ? idx_r[row - kn] : row - kn;
      v = c * P[a * n_r + b];
    }
    A[idx] = v;
  }
}

__global__ void export_kernel(int64_t n_ns, int64_t n_r, const uint8_t* __restrict__ M_ns,
                              const uint8_t* __restrict__ M_r, const double* __restrict__ P,
                              const double* __restrict__ c0, double2* __restrict__ X) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_ns * n_r; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx / n_r, b = idx - a * n_r;
    X[idx] = xval(c0, P[idx], M_ns[a] + M_r[b]);
  }
}

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  return (int)(g < 152 * 32 ? (g < 1 ? 1 : g) : 152 * 32);
}

}  // namespace

tgba_status assemble_heff(Basis& b, double h_x, double* heff, cudaStream_t st) {
  const double scale = -b.L * h_x;
  for (const Sector& sec : b.sectors) {
    const int64_t n = sec.n_ns + sec.n_r;
    if (n == 0) continue;
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    heff_kernel<<<grid, block, 0, st>>>(sec.n_ns, sec.n_r, b.d_E_ns + sec.ns_off, b.d_E_r + sec.r_off,
                                        b.d_M_ns + sec.ns_off, b.d_M_r + sec.r_off, b.d_P + sec.x_off, b.d_c0, scale,
                                        (double2*)heff + sec.h_off);
    TGBA_CUDA(cudaGetLastError());
    ++b.launches;
  }
  return TGBA_OK;
}

tgba_status export_x(Basis& b, int s, double* x, cudaStream_t st) {
  const Sector& sec = b.sectors[s];
  const int64_t work = sec.n_ns * sec.n_r;
  if (work == 0) return TGBA_OK;
  export_kernel<<<grid_for(work, 256), 256, 0, st>>>(sec.n_ns, sec.n_r, b.d_M_ns + sec.ns_off, b.d_M_r + sec.r_off,
                                                     b.d_P + sec.x_off, b.d_c0, (double2*)x);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

tgba_status build_real_heff(Basis& b, int s, double h_x, double* a, const int32_t* idx_ns, int64_t kn,
                            const int32_t* idx_r, int64_t kr, cudaStream_t st) {
  const Sector& sec = b.sectors[s];
  const int64_t n = kn + kr;
  if (n == 0) return TGBA_OK;
  heff_real_kernel<<<grid_for(n * n, 256), 256, 0, st>>>(kn, kr, idx_ns, idx_r, sec.n_r, b.d_E_ns + sec.ns_off,
                                                         b.d_E_r + sec.r_off, b.d_P + sec.x_off, b.d_c0,
                                                         -b.L * h_x, a);
  TGBA_CUDA(cudaGetLastError());
  ++b.launches;
  return TGBA_OK;
}

}  // namespace tgba
