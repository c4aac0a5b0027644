// Host set-up, part 4: the near-element correction of Eq. 14c.
// Sources are tetrahedra (uniform rho_e = -sum_j M_j . grad(phi_j)) and true boundary
// triangles (linear sigma = M . n).  Their point charges (Eq. 14b) are the nodal moments
// rho_e V_e / 4 and (A/12)(2 sigma_k + sum_{j != k} sigma_j).  For every placement of an
// element (translated by a lattice vector l) that is near observer n -- a vertex lands on
// the node, or its centroid lies within r_E = near_elem_factor * mean edge -- the exact
// integral replaces the point charges:
//   4 pi u_n += int_{s+l} G0(r_n - r') dens_s - sum_k q_k^s G0'(r_n - r_k - l),  G0'(0) = 0.
// The result is linear in M and is stored per (n, k) as a 3-vector: on the adjacency
// pattern when k is a neighbour of n (always so for touching elements), otherwise in a
// separate sparse matrix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <unordered_map>

#include "internal.hpp"

namespace pmfem {

namespace {
struct Placement {
  int64_t elem;   // tet index, or T + boundary-face index
  int32_t img[3];
};
bool operator<(const Placement& a, const Placement& b) {
  if (a.elem != b.elem) return a.elem < b.elem;
  for (int d = 0; d < 3; ++d)
    if (a.img[d] != b.img[d]) return a.img[d] < b.img[d];
  return false;
}
bool operator==(const Placement& a, const Placement& b) {
  return a.elem == b.elem && a.img[0] == b.img[0] && a.img[1] == b.img[1] && a.img[2] == b.img[2];
}
}  // namespace

int setup_near_elements(Setup& s, Error& err) {
  (void)err;
  const int64_t Np = s.Np, T = s.T, F = (int64_t)s.bfaces.size() / 3;
  const double rE = s.near_elem_factor * s.mean_edge;
  const double self_tol = 1e-6 * s.mean_edge;
  // incidence of unknowns in tetrahedra and boundary triangles
  std::vector<int64_t> ptr(Np + 1, 0);
  for (int64_t i = 0; i < 4 * T; ++i) ptr[s.lca[s.tets[i]] + 1]++;
  for (int64_t i = 0; i < 3 * F; ++i) ptr[s.lca[s.bfaces[i]] + 1]++;
  for (int64_t u = 0; u < Np; ++u) ptr[u + 1] += ptr[u];
  std::vector<int64_t> inc(ptr[Np]), fill(ptr.begin(), ptr.end() - 1);
  for (int64_t i = 0; i < 4 * T; ++i) inc[fill[s.lca[s.tets[i]]]++] = i;                 // tet slot
  for (int64_t i = 0; i < 3 * F; ++i) inc[fill[s.lca[s.bfaces[i]]]++] = 4 * T + i;       // face slot
  // element centroids and bounding info for the radius search
  const int64_t nel = T + F;
  std::vector<double> cen;
  std::unordered_map<int64_t, std::vector<int64_t>> cells;
  double cell = 0;
  int span[3] = {0, 0, 0};
  auto cell_key = [](int64_t a, int64_t b, int64_t c) {
    return (a * 73856093LL) ^ (b * 19349663LL) ^ (c * 83492791LL);
  };
  if (rE > 0) {
    cen.resize(3 * nel);
    for (int64_t e = 0; e < T; ++e)
      for (int d = 0; d < 3; ++d) {
        double acc = 0;
        for (int i = 0; i < 4; ++i) acc += s.xyz[3 * (int64_t)s.tets[4 * e + i] + d];
        cen[3 * e + d] = acc / 4.0;
      }
    for (int64_t f = 0; f < F; ++f)
      for (int d = 0; d < 3; ++d) {
        double acc = 0;
        for (int i = 0; i < 3; ++i) acc += s.xyz[3 * (int64_t)s.bfaces[3 * f + i] + d];
        cen[3 * (T + f) + d] = acc / 3.0;
      }
    cell = rE;
    for (int64_t e = 0; e < nel; ++e) {
      int64_t k = cell_key((int64_t)std::floor(cen[3 * e] / cell), (int64_t)std::floor(cen[3 * e + 1] / cell),
                           (int64_t)std::floor(cen[3 * e + 2] / cell));
      cells[k].push_back(e);
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < s.N; ++i)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], s.xyz[3 * i + d]);
        hi[d] = std::max(hi[d], s.xyz[3 * i + d]);
      }
    for (int d = 0; d < 3; ++d) span[d] = s.periodic[d] ? (int)std::ceil((hi[d] - lo[d]) / s.L[d]) + 2 : 0;
  }

  const int64_t nnz = s.rowptr[Np];
  s.Ea.assign(3 * nnz, 0.0);
  std::vector<std::vector<std::pair<int32_t, std::array<double, 3>>>> extra(Np);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    std::vector<Placement> pl;
    std::map<int32_t, std::array<double, 3>> ext;
    for (int64_t n = b; n < e; ++n) {
      const double* rn = &s.pos_f[3 * n];
      pl.clear();
      ext.clear();
      // (a) elements with a vertex on the node
      for (int64_t t = ptr[n]; t < ptr[n + 1]; ++t) {
        int64_t slot = inc[t];
        int32_t v = slot < 4 * T ? s.tets[slot] : s.bfaces[slot - 4 * T];
        Placement P;
        P.elem = slot < 4 * T ? slot / 4 : T + (slot - 4 * T) / 3;
        for (int d = 0; d < 3; ++d)
          P.img[d] = s.periodic[d] ? (int32_t)std::nearbyint((rn[d] - s.xyz[3 * (int64_t)v + d]) / s.L[d]) : 0;
        pl.push_back(P);
      }
      // (b) elements whose centroid lies within r_E (all lattice placements)
      if (rE > 0) {
        for (int ix = -span[0]; ix <= span[0]; ++ix)
          for (int iy = -span[1]; iy <= span[1]; ++iy)
            for (int iz = -span[2]; iz <= span[2]; ++iz) {
              double q[3] = {rn[0] - ix * s.L[0], rn[1] - iy * s.L[1], rn[2] - iz * s.L[2]};
              int64_t c0 = (int64_t)std::floor(q[0] / cell), c1 = (int64_t)std::floor(q[1] / cell),
                      c2 = (int64_t)std::floor(q[2] / cell);
              for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                  for (int dz = -1; dz <= 1; ++dz) {
                    auto it = cells.find(cell_key(c0 + dx, c1 + dy, c2 + dz));
                    if (it == cells.end()) continue;
                    for (int64_t el : it->second) {
                      const double* c = &cen[3 * el];
                      // the hash may collide: check the cell and the distance exactly
                      if ((int64_t)std::floor(c[0] / cell) != c0 + dx || (int64_t)std::floor(c[1] / cell) != c1 + dy ||
                          (int64_t)std::floor(c[2] / cell) != c2 + dz)
                        continue;
                      double d0 = c[0] - q[0], d1 = c[1] - q[1], d2 = c[2] - q[2];
                      if (d0 * d0 + d1 * d1 + d2 * d2 <= rE * rE) pl.push_back({el, {ix, iy, iz}});
                    }
                  }
            }
      }
      std::sort(pl.begin(), pl.end());
      pl.erase(std::unique(pl.begin(), pl.end()), pl.end());
      auto add = [&](int32_t k, const double v[3]) {
        const int32_t* cb = s.col.data() + s.rowptr[n];
        const int32_t* ce = s.col.data() + s.rowptr[n + 1];
        const int32_t* it = std::lower_bound(cb, ce, k);
        if (it != ce && *it == k) {
          int64_t pos = it - s.col.data();
          for (int d = 0; d < 3; ++d) s.Ea[3 * pos + d] += v[d];
        } else {
          auto& a = ext[k];
          for (int d = 0; d < 3; ++d) a[d] += v[d];
        }
      };
      for (const Placement& P : pl) {
        double obs[3];
        for (int d = 0; d < 3; ++d) obs[d] = rn[d] - P.img[d] * s.L[d];
        if (P.elem < T) {
          double X[4][3], g[4][3];
          int32_t vid[4];
          for (int i = 0; i < 4; ++i) {
            vid[i] = s.tets[4 * P.elem + i];
            for (int d = 0; d < 3; ++d) X[i][d] = s.xyz[3 * (int64_t)vid[i] + d];
          }
          double Ve = tet_grads(X, g);
          double I = tet_potential(obs, X);
          double Ppt = 0;
          for (int i = 0; i < 4; ++i) {
            double d0 = obs[0] - X[i][0], d1 = obs[1] - X[i][1], d2 = obs[2] - X[i][2];
            double dist = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            bool self = s.lca[vid[i]] == n && dist < self_tol;
            if (!self) Ppt += 0.25 * Ve / dist;
          }
          const double coef = I - Ppt;
          for (int j = 0; j < 4; ++j) {
            double v[3] = {-g[j][0] * coef, -g[j][1] * coef, -g[j][2] * coef};
            add(s.lca[vid[j]], v);
          }
        } else {
          const int64_t f = P.elem - T;
          int32_t vid[3];
          double X[3][3];
          for (int i = 0; i < 3; ++i) {
            vid[i] = s.bfaces[3 * f + i];
            for (int d = 0; d < 3; ++d) X[i][d] = s.xyz[3 * (int64_t)vid[i] + d];
          }
          double e1[3] = {X[1][0] - X[0][0], X[1][1] - X[0][1], X[1][2] - X[0][2]};
          double e2[3] = {X[2][0] - X[0][0], X[2][1] - X[0][1], X[2][2] - X[0][2]};
          double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
          double a2 = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
          double nrm[3] = {nn[0] / a2, nn[1] / a2, nn[2] / a2};
          const double area = 0.5 * a2;
          double Ij[3];
          tri_hat_potentials(obs, X[0], X[1], X[2], Ij);
          double G[3], Gs = 0;
          for (int i = 0; i < 3; ++i) {
            double d0 = obs[0] - X[i][0], d1 = obs[1] - X[i][1], d2 = obs[2] - X[i][2];
            double dist = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            bool self = s.lca[vid[i]] == n && dist < self_tol;
            G[i] = self ? 0.0 : 1.0 / dist;
            Gs += G[i];
          }
          for (int j = 0; j < 3; ++j) {
            double coef = Ij[j] - area / 12.0 * (Gs + G[j]);
            double v[3] = {nrm[0] * coef, nrm[1] * coef, nrm[2] * coef};
            add(s.lca[vid[j]], v);
          }
        }
      }
      for (auto& kv : ext) extra[n].push_back({kv.first, kv.second});
    }
  }, 64);
  for (auto& x : s.Ea) x *= s.Ms;
  s.Ex.rows = Np;
  s.Ex.comps = 3;
  s.Ex.rowptr.assign(Np + 1, 0);
  for (int64_t n = 0; n < Np; ++n) s.Ex.rowptr[n + 1] = s.Ex.rowptr[n] + (int32_t)extra[n].size();
  s.Ex.col.resize(s.Ex.rowptr[Np]);
  s.Ex.vals.resize(3 * (size_t)s.Ex.rowptr[Np]);
  for (int64_t n = 0; n < Np; ++n)
    for (size_t i = 0; i < extra[n].size(); ++i) {
      int64_t o = s.Ex.rowptr[n] + i;
      s.Ex.col[o] = extra[n][i].first;
      for (int d = 0; d < 3; ++d) s.Ex.vals[3 * o + d] = s.Ms * extra[n][i].second[d];
    }
  return OK;
}

int run_setup(Setup& s, Error& err) {
  int rc;
  s.ready = false;
  auto t0 = std::chrono::steady_clock::now();
  auto lap = [&](int i) {
    auto t1 = std::chrono::steady_clock::now();
    s.t_stage[i] = std::chrono::duration<double>(t1 - t0).count();
    t0 = t1;
  };
  if ((rc = setup_pairing(s, err))) return rc;
  lap(0);
  if ((rc = setup_operators(s, err))) return rc;
  lap(1);
  if ((rc = setup_grid(s, err))) return rc;
  lap(2);
  if ((rc = setup_spectrum(s, err))) return rc;
  lap(3);
  if ((rc = setup_near_elements(s, err))) return rc;
  lap(4);
  if ((rc = setup_precorrection(s, err))) return rc;
  lap(5);
  s.ready = true;
  return OK;
}

}  // namespace pmfem
