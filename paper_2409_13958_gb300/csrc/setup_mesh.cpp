// Host set-up, part 1: mesh checks, periodic pairing with LCA (Sec. 2.2), the protruding
// fold (Eq. 18) and the periodized P1 operators (Eqs. 7-12, 14a, 14d).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "internal.hpp"

namespace pmfem {

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f, int64_t min_chunk) {
  if (n <= 0) return;
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int64_t nt = std::min<int64_t>(hw, (n + min_chunk - 1) / min_chunk);
  if (nt <= 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back(f, b, e);
  }
  for (auto& x : th) x.join();
}

static inline void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static inline void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Volume (signed) and gradients of the four barycentric coordinates.
double tet_grads(const double X[4][3], double g[4][3]) { return sm::tet_grads(X, g); }

static void load_tet(const Setup& s, int64_t e, double X[4][3]) {
  for (int i = 0; i < 4; ++i) {
    int32_t v = s.tets[4 * e + i];
    for (int d = 0; d < 3; ++d) X[i][d] = s.xyz[3 * (int64_t)v + d];
  }
}

int setup_validate_mesh(Setup& s, Error& err) {
  if (s.N > (int64_t(1) << 30)) {   // device kernels index columns in int32 with a modular wrap
    err = {EINVAL_, "more than 2^30 nodes"};
    return EINVAL_;
  }
  for (int64_t i = 0; i < 4 * s.T; ++i) {
    if (s.tets[i] < 0 || s.tets[i] >= s.N) {
      err = {EMESH_, "tetrahedron " + std::to_string(i / 4) + " has a node index outside [0, N)"};
      return EMESH_;
    }
  }
  for (int64_t i = 0; i < 3 * s.N; ++i) {
    if (!std::isfinite(s.xyz[i])) {
      err = {EMESH_, "node coordinate " + std::to_string(i / 3) + " is not finite"};
      return EMESH_;
    }
  }
  int64_t bad = -1;
  for (int64_t e = 0; e < s.T; ++e) {
    double X[4][3], g[4][3];
    load_tet(s, e, X);
    double V = tet_grads(X, g);
    double lmax = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double d[3];
        sub3(X[a], X[b], d);
        lmax = std::max(lmax, std::sqrt(dot3(d, d)));
      }
    if (!(std::fabs(6.0 * V) > 1e-12 * lmax * lmax * lmax)) {
      bad = e;
      break;
    }
    if (V < 0) std::swap(s.tets[4 * e + 2], s.tets[4 * e + 3]);
  }
  if (bad >= 0) {
    err = {EMESH_, "tetrahedron " + std::to_string(bad) + " is degenerate"};
    return EMESH_;
  }
  return OK;
}

// ------------------------------------------------------------------------------------
// PBC pairs: nodes i, j with r_j - r_i = sum n_a L_a e_a, n_a in {-1,0,1}, not all 0,
// found through a hash of quantised coordinates; chains merged by union-find; the
// ancestor of a group is its member with the lexicographically smallest periodic
// coordinates; unknowns numbered by increasing original node index.
// ------------------------------------------------------------------------------------
namespace {
struct Key3 {
  int64_t a, b, c;
  bool operator==(const Key3& o) const { return a == o.a && b == o.b && c == o.c; }
};
struct Key3Hash {
  size_t operator()(const Key3& k) const {
    uint64_t h = (uint64_t)k.a * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k.b + 0x7F4A7C159E3779B9ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.c + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};
int64_t uf_find(std::vector<int64_t>& p, int64_t i) {
  while (p[i] != i) {
    p[i] = p[p[i]];
    i = p[i];
  }
  return i;
}
}  // namespace

int setup_pairing(Setup& s, Error& err) {
  const int64_t N = s.N;
  std::vector<int64_t> parent(N);
  std::iota(parent.begin(), parent.end(), 0);
  int per[3], np = 0;
  double Lmin = 0;
  for (int a = 0; a < 3; ++a) {
    s.periodic[a] = s.L[a] > 0;
    if (s.periodic[a]) {
      per[np++] = a;
      Lmin = (np == 1) ? s.L[a] : std::min(Lmin, s.L[a]);
    }
  }
  std::vector<char> on_face(N, 0);
  if (np > 0) {
    const double tol = 1e-9 * Lmin;
    const double cell = 4.0 * tol;
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = 1e300;
      hi[d] = -1e300;
    }
    for (int64_t i = 0; i < N; ++i)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], s.xyz[3 * i + d]);
        hi[d] = std::max(hi[d], s.xyz[3 * i + d]);
      }
    std::unordered_map<Key3, std::vector<int32_t>, Key3Hash> grid;
    grid.reserve((size_t)N * 2);
    for (int64_t i = 0; i < N; ++i) {
      const double* x = &s.xyz[3 * i];
      Key3 k{(int64_t)std::floor(x[0] / cell), (int64_t)std::floor(x[1] / cell), (int64_t)std::floor(x[2] / cell)};
      grid[k].push_back((int32_t)i);
    }
    int noff = 1;
    for (int t = 0; t < np; ++t) noff *= 3;
    for (int64_t i = 0; i < N; ++i) {
      const double* x = &s.xyz[3 * i];
      for (int o = 0; o < noff; ++o) {
        int code = o, nz = 0;
        double tgt[3] = {x[0], x[1], x[2]};
        for (int t = 0; t < np; ++t) {
          int n = code % 3 - 1;
          code /= 3;
          if (n) nz = 1;
          tgt[per[t]] += n * s.L[per[t]];
        }
        if (!nz) continue;
        bool inside = true;
        for (int d = 0; d < 3; ++d)
          if (tgt[d] < lo[d] - tol || tgt[d] > hi[d] + tol) inside = false;
        if (!inside) continue;
        int64_t c0 = (int64_t)std::floor(tgt[0] / cell), c1 = (int64_t)std::floor(tgt[1] / cell),
                c2 = (int64_t)std::floor(tgt[2] / cell);
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
              auto it = grid.find(Key3{c0 + dx, c1 + dy, c2 + dz});
              if (it == grid.end()) continue;
              for (int32_t j : it->second) {
                const double* y = &s.xyz[3 * (int64_t)j];
                double d0 = y[0] - tgt[0], d1 = y[1] - tgt[1], d2 = y[2] - tgt[2];
                if (d0 * d0 + d1 * d1 + d2 * d2 <= tol * tol) {
                  int64_t ri = uf_find(parent, i), rj = uf_find(parent, j);
                  if (ri != rj) parent[std::max(ri, rj)] = std::min(ri, rj);
                  on_face[i] = on_face[j] = 1;
                }
              }
            }
      }
    }
  }
  // ancestor of each group: lexicographically smallest periodic coordinates
  std::vector<int64_t> comp(N), anc(N, -1);
  for (int64_t i = 0; i < N; ++i) comp[i] = uf_find(parent, i);
  auto less_per = [&](int64_t a, int64_t b) {
    for (int t = 0; t < np; ++t) {
      double xa = s.xyz[3 * a + per[t]], xb = s.xyz[3 * b + per[t]];
      if (xa != xb) return xa < xb;
    }
    return a < b;
  };
  for (int64_t i = 0; i < N; ++i) {
    int64_t c = comp[i];
    if (anc[c] < 0 || less_per(i, anc[c])) anc[c] = i;
  }
  std::vector<int32_t> uid(N, -1);
  s.roots.clear();
  for (int64_t i = 0; i < N; ++i)
    if (anc[comp[i]] == i) {
      uid[i] = (int32_t)s.roots.size();
      s.roots.push_back((int32_t)i);
    }
  s.Np = (int64_t)s.roots.size();
  s.lca.assign(N, 0);
  for (int64_t i = 0; i < N; ++i) s.lca[i] = uid[anc[comp[i]]];
  // touching faces must conform: along a periodic axis with pairs, every node lying on
  // the extreme coordinate planes of that axis needs a partner
  for (int t = 0; t < np; ++t) {
    int a = per[t];
    double lo = 1e300, hi = -1e300;
    for (int64_t i = 0; i < N; ++i) {
      lo = std::min(lo, s.xyz[3 * i + a]);
      hi = std::max(hi, s.xyz[3 * i + a]);
    }
    if (std::fabs((hi - lo) - s.L[a]) > 1e-9 * s.L[a]) continue;   // not a flat touching cell
    int64_t paired = 0, lonely = -1;
    for (int64_t i = 0; i < N; ++i) {
      double x = s.xyz[3 * i + a];
      bool face = std::fabs(x - lo) <= 1e-9 * s.L[a] || std::fabs(x - hi) <= 1e-9 * s.L[a];
      if (!face) continue;
      if (on_face[i]) ++paired;
      else if (lonely < 0) lonely = i;
    }
    if (paired > 0 && lonely >= 0) {
      err = {EMESH_, "node " + std::to_string(lonely) + " lies on a touching periodic face but has no periodic partner"};
      return EMESH_;
    }
  }
  // fold (Eq. 18): window [r0 - L/2, r0 + L/2) about the mean of the unknowns
  s.pos_f.assign(3 * s.Np, 0.0);
  for (int d = 0; d < 3; ++d) {
    double acc = 0;
    for (int64_t u = 0; u < s.Np; ++u) acc += s.xyz[3 * (int64_t)s.roots[u] + d];
    s.r0[d] = acc / (double)s.Np;
  }
  for (int64_t u = 0; u < s.Np; ++u)
    for (int d = 0; d < 3; ++d) {
      double x = s.xyz[3 * (int64_t)s.roots[u] + d];
      if (s.periodic[d]) {
        double k = std::floor((x - s.r0[d] + 0.5 * s.L[d]) / s.L[d]);
        x = x - k * s.L[d];
      }
      s.pos_f[3 * u + d] = x;
    }
  return OK;
}

}  // namespace pmfem
