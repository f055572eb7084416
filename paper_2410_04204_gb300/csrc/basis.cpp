// Host side of the basis: single-particle modes (Eq. 6-7, S3), enumeration and truncation of
// the Gaussian basis per momentum sector (Method section, Appendix B), and the tiling of the
// NS x R pair grid into work units of uniform Pfaffian size.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "tgba_internal.h"

namespace tgba {

// Size classes of the Pfaffian kernels.  Classes 0..7: exact n = 0, 2, ..., 14 (register
// kernel, 128 threads); classes 8..11: n <= 16, 20, 24, 32 (shared-memory kernel).
int tile_class(int n) {
  if (n <= 14) return n / 2;
  if (n <= 16) return 8;
  if (n <= 20) return 9;
  if (n <= 24) return 10;
  return 11;
}

Modes make_modes(int N, int parity, double h) {
  Modes md;
  md.N = N; md.parity = parity; md.h = h;
  md.nlab.resize(N); md.eps.resize(N); md.theta.resize(N); md.ex.resize(N);
  const double pi = M_PI;
  for (int i = 0; i < N; ++i) {
    int n = (parity == 0 ? -(N - 1) : -(N - 2)) + 2 * i;
    md.nlab[i] = n;
    double k = pi * n / N;
    if (n == N) {
      md.eps[i] = 2.0 * (h - 1.0);       // signed at k = pi (Eq. 7)
      md.theta[i] = 0.0;                 // 2(h-1)/eps_pi = 1, taken also at h = 1
      md.ex[i] = -md.eps[i];             // removing the d_pi quasiparticle of |0>_R
    } else {
      double c = std::cos(0.5 * k);
      md.eps[i] = 2.0 * std::sqrt((h - 1.0) * (h - 1.0) + 4.0 * h * c * c);
      if (n == 0) {
        md.theta[i] = 0.0;               // sign(0) = 0
      } else {
        double x = 2.0 * (h + std::cos(k)) / md.eps[i];
        x = std::min(1.0, std::max(-1.0, x));
        md.theta[i] = std::copysign(std::acos(x), k);
      }
      md.ex[i] = md.eps[i];
    }
  }
  double s = 0.0;
  for (int i = 0; i < N; ++i)
    if (md.nlab[i] != N) s += md.eps[i];
  md.e_vac = -0.5 * s;
  if (parity == 1) md.e_vac += 0.5 * md.eps[N - 1];
  double norm = 1.0;
  for (int i = 0; i < N; ++i)
    if (md.nlab[i] > 0 && md.nlab[i] != N) norm /= std::cos(0.5 * md.theta[i]);
  md.norm = norm;
  return md;
}

namespace {

struct Found {
  double E;
  int M;
  int16_t modes[kMaxQp];
};

bool key_emm(const Found& a, const Found& b) {   // (E, M, modes)
  if (a.E != b.E) return a.E < b.E;
  if (a.M != b.M) return a.M < b.M;
  return std::lexicographical_compare(a.modes, a.modes + a.M, b.modes, b.modes + b.M);
}

bool key_mem(const Found& a, const Found& b) {   // (M, E, modes): basis order
  if (a.M != b.M) return a.M < b.M;
  if (a.E != b.E) return a.E < b.E;
  return std::lexicographical_compare(a.modes, a.modes + a.M, b.modes, b.modes + b.M);
}

// All states of one parity, binned by sector.  Depth-first over the modes in ascending
// excitation energy; a branch is cut when even the most negative completion exceeds the cutoff.
tgba_status enumerate_parity(const Modes& md, int max_qp, double cut, const std::vector<int>& sector_of_m,
                             std::vector<std::vector<Found>>& out) {
  const int N = md.N;
  std::vector<int> order(N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return md.ex[a] < md.ex[b]; });
  std::vector<double> neg_suffix(N + 1, 0.0);
  for (int t = N - 1; t >= 0; --t) neg_suffix[t] = neg_suffix[t + 1] + std::min(0.0, md.ex[order[t]]);
  int chosen[kMaxQp];
  int depth = 0;
  int64_t visited = 0;
  const int64_t kVisitLimit = 2000000000LL;
  bool over = false;
  std::function<void(int, double, int)> dfs = [&](int t, double e_part, int nsum) {
    if (over) return;
    if (++visited > kVisitLimit) { over = true; return; }
    if (md.e_vac + e_part + neg_suffix[t] > cut + 1e-6) return;
    if (depth % 2 == 0) {
      int r = ((nsum % (2 * N)) + 2 * N) % (2 * N);
      int s = sector_of_m[r / 2];
      if (s >= 0) {
        Found f;
        f.M = depth;
        double ex[kMaxQp];
        for (int q = 0; q < depth; ++q) { f.modes[q] = (int16_t)chosen[q]; ex[q] = md.ex[chosen[q]]; }
        std::sort(f.modes, f.modes + depth);
        std::sort(ex, ex + depth);
        double sum = 0.0;                      // canonical: ascending values, from 0
        for (int q = 0; q < depth; ++q) sum += ex[q];
        f.E = md.e_vac + sum;
        if (f.E <= cut) out[s].push_back(f);
      }
    }
    if (depth == max_qp) return;
    for (int u = t; u < N; ++u) {
      int i = order[u];
      chosen[depth++] = i;
      dfs(u + 1, e_part + md.ex[i], nsum + md.nlab[i]);
      --depth;
    }
  };
  dfs(0, 0.0, 0);
  if (over) return fail(TGBA_ELIMIT, "basis enumeration visited more than 2e9 states; tighten max_qp or e_cut");
  return TGBA_OK;
}

}  // namespace

tgba_status enumerate_basis(const tgba_model& model, const int32_t* sectors, int n_sectors, const tgba_trunc& tr,
                            Basis& b) {
  const int N = model.L;
  b.L = N;
  b.J = model.J;
  b.h = model.h_z / model.J;
  b.max_qp = tr.max_qp;
  b.e_cut = tr.e_cut;
  b.cap = tr.max_per_parity;
  Modes mns = make_modes(N, 0, b.h), mr = make_modes(N, 1, b.h);
  b.e_ns_vac = mns.e_vac;
  // energies in units of J: the cutoff is given in absolute units
  double cut = tr.e_cut >= 0 ? (mns.e_vac + tr.e_cut / model.J) + 1e-9 / model.J : INFINITY;
  std::vector<int> sector_of_m(N, -1);
  for (int s = 0; s < n_sectors; ++s) sector_of_m[sectors[s]] = s;
  std::vector<std::vector<Found>> fns(n_sectors), fr(n_sectors);
  tgba_status st = enumerate_parity(mns, tr.max_qp, cut, sector_of_m, fns);
  if (st != TGBA_OK) return st;
  st = enumerate_parity(mr, tr.max_qp, cut, sector_of_m, fr);
  if (st != TGBA_OK) return st;

  b.sectors.assign(n_sectors, Sector());
  int64_t x_off = 0, h_off = 0, ev_off = 0;
  int max_n = 0;
  for (int s = 0; s < n_sectors; ++s) {
    Sector& sec = b.sectors[s];
    sec.m = sectors[s];
    for (int p = 0; p < 2; ++p) {
      std::vector<Found>& v = p == 0 ? fns[s] : fr[s];
      std::sort(v.begin(), v.end(), key_emm);
      if (tr.max_per_parity > 0 && (int64_t)v.size() > tr.max_per_parity) v.resize(tr.max_per_parity);
      std::sort(v.begin(), v.end(), key_mem);
      StateTable& T = p == 0 ? b.ns : b.r;
      int64_t off = (int64_t)T.E.size();
      std::vector<Group>& G = p == 0 ? sec.g_ns : sec.g_r;
      for (size_t q = 0; q < v.size(); ++q) {
        T.E.push_back(v[q].E * model.J);
        T.M.push_back((uint8_t)v[q].M);
        for (int z = 0; z < tr.max_qp; ++z) T.modes.push_back(z < v[q].M ? v[q].modes[z] : (int16_t)-1);
        if (G.empty() || G.back().M != v[q].M) G.push_back(Group{v[q].M, off + (int64_t)q, off + (int64_t)q + 1});
        else G.back().end = off + (int64_t)q + 1;
      }
      for (Group& g : G) { g.begin -= off; g.end -= off; }   // sector-relative
      if (p == 0) { sec.ns_off = off; sec.n_ns = (int64_t)v.size(); }
      else { sec.r_off = off; sec.n_r = (int64_t)v.size(); }
    }
    if (sec.n_ns * sec.n_r >= (int64_t)1 << 31)
      return fail(TGBA_ELIMIT, "a sector has more than 2^31 NS x R elements");
    sec.x_off = x_off; x_off += sec.n_ns * sec.n_r;
    int64_t n = sec.n_ns + sec.n_r;
    sec.h_off = h_off; h_off += n * n;
    sec.ev_off = ev_off; ev_off += n;
    int mn = sec.g_ns.empty() ? 0 : sec.g_ns.back().M, mr_ = sec.g_r.empty() ? 0 : sec.g_r.back().M;
    if (!sec.g_ns.empty() && !sec.g_r.empty()) max_n = std::max(max_n, mn + mr_);
  }
  b.n_elements = x_off;
  b.n_heff = h_off;
  b.n_states = ev_off;
  b.max_n = max_n;
  return TGBA_OK;
}

void build_rects(Basis& b) {
  b.rect_lists.assign(kNumClasses, RectList());
  for (int c = 0; c < kNumClasses; ++c) b.rect_lists[c].nmax = c < 8 ? 2 * c : c == 8 ? 16 : c == 9 ? 20 : c == 10 ? 24 : 32;
  for (size_t s = 0; s < b.sectors.size(); ++s) {
    const Sector& sec = b.sectors[s];
    for (const Group& ga : sec.g_ns)
      for (const Group& gb : sec.g_r) {
        Rect r;
        r.out0 = sec.x_off + ga.begin * sec.n_r + gb.begin;
        r.ns0 = sec.ns_off + ga.begin;
        r.r0 = sec.r_off + gb.begin;
        r.ld = (int32_t)sec.n_r;
        r.w = (int32_t)(gb.end - gb.begin);
        r.rows = (int32_t)(ga.end - ga.begin);
        r.n = ga.M + gb.M;
        r.Ma = ga.M;
        r.pad = 0;
        r.tile0 = 0;
        b.rect_lists[tile_class(r.n)].rects.push_back(r);
      }
  }
  std::vector<Rect> all_reg;
  b.max_reg_n = 0;
  for (int c = 0; c < kNumClasses; ++c) {
    RectList& Lc = b.rect_lists[c];
    std::stable_sort(Lc.rects.begin(), Lc.rects.end(), [](const Rect& x, const Rect& y) { return x.n > y.n; });
    int64_t t = 0;
    for (Rect& r : Lc.rects) {
      r.tile0 = t;
      t += ((int64_t)r.rows * r.w + 31) / 32;
    }
    Lc.n_tiles = t;
    Lc.n_rects = (int)Lc.rects.size();
    if (Lc.nmax <= 14)
      for (const Rect& r : Lc.rects) {
        all_reg.push_back(r);
        b.max_reg_n = std::max(b.max_reg_n, r.n);
      }
  }
  std::stable_sort(all_reg.begin(), all_reg.end(), [](const Rect& x, const Rect& y) { return x.n > y.n; });
  int64_t t = 0;
  for (Rect& r : all_reg) {
    r.tile0 = t;
    t += ((int64_t)r.rows * r.w + 31) / 32;
  }
  b.reg_tiles_total = t;
  b.reg_rects_total = (int)all_reg.size();
  b.reg_rects = all_reg;
}

}  // namespace tgba
