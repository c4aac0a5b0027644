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

  // phase 1 (host): the near placements of every row, sorted, and for every vertex of a
  // placement its output slot: the adjacency position when the vertex's unknown is a
  // neighbour of the row, else a slot among the row's extra columns (sorted, after nnz)
  const int64_t nnz = s.rowptr[Np];
  std::vector<std::vector<Placement>> rows_pl(Np);
  std::vector<std::vector<int32_t>> rows_x(Np);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e; ++n) {
      const double* rn = &s.pos_f[3 * n];
      std::vector<Placement>& pl = rows_pl[n];
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
      // columns outside the adjacency pattern (only elements found by the radius reach them)
      std::vector<int32_t>& xc = rows_x[n];
      const int32_t* cb = s.col.data() + s.rowptr[n];
      const int32_t* ce = s.col.data() + s.rowptr[n + 1];
      for (const Placement& P : pl) {
        const int nv = P.elem < T ? 4 : 3;
        for (int j = 0; j < nv; ++j) {
          const int32_t v = P.elem < T ? s.tets[4 * P.elem + j] : s.bfaces[3 * (P.elem - T) + j];
          const int32_t k = s.lca[v];
          const int32_t* it = std::lower_bound(cb, ce, k);
          if (!(it != ce && *it == k)) xc.push_back(k);
        }
      }
      std::sort(xc.begin(), xc.end());
      xc.erase(std::unique(xc.begin(), xc.end()), xc.end());
    }
  }, 64);
  NearPlan plan;
  plan.pptr.assign(Np + 1, 0);
  plan.xptr.assign(Np + 1, 0);
  for (int64_t n = 0; n < Np; ++n) {
    plan.pptr[n + 1] = plan.pptr[n] + (int64_t)rows_pl[n].size();
    plan.xptr[n + 1] = plan.xptr[n] + (int64_t)rows_x[n].size();
  }
  const int64_t npl = plan.pptr[Np], nx = plan.xptr[Np];
  plan.elem.resize(npl);
  plan.img.resize(3 * npl);
  plan.dest.assign(4 * npl, 0);
  plan.xcol.resize(nx);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    for (int64_t n = b; n < e; ++n) {
      const int32_t* cb = s.col.data() + s.rowptr[n];
      const int32_t* ce = s.col.data() + s.rowptr[n + 1];
      const std::vector<int32_t>& xc = rows_x[n];
      std::copy(xc.begin(), xc.end(), plan.xcol.begin() + plan.xptr[n]);
      int64_t q = plan.pptr[n];
      for (const Placement& P : rows_pl[n]) {
        plan.elem[q] = P.elem;
        for (int d = 0; d < 3; ++d) plan.img[3 * q + d] = P.img[d];
        const int nv = P.elem < T ? 4 : 3;
        for (int j = 0; j < nv; ++j) {
          const int32_t v = P.elem < T ? s.tets[4 * P.elem + j] : s.bfaces[3 * (P.elem - T) + j];
          const int32_t k = s.lca[v];
          const int32_t* it = std::lower_bound(cb, ce, k);
          if (it != ce && *it == k) {
            plan.dest[4 * q + j] = (int64_t)(it - s.col.data());
          } else {
            const int64_t xi = std::lower_bound(xc.begin(), xc.end(), k) - xc.begin();
            plan.dest[4 * q + j] = nnz + plan.xptr[n] + xi;
          }
        }
        ++q;
      }
      std::vector<Placement>().swap(rows_pl[n]);
      std::vector<int32_t>().swap(rows_x[n]);
    }
  }, 64);
  // phase 2: the integrals, row by row (host threads, or one GPU thread per row), into
  // 3 x (nnz + extra) values
  sm::NearArgs A;
  A.xyz = s.xyz.data();
  A.tets = s.tets.data();
  A.bfaces = s.bfaces.data();
  A.lca = s.lca.data();
  A.pos_f = s.pos_f.data();
  for (int d = 0; d < 3; ++d) A.L[d] = s.periodic[d] ? s.L[d] : 0.0;
  A.T = T;
  A.self_tol = self_tol;
  A.pptr = plan.pptr.data();
  A.elem = plan.elem.data();
  A.img = plan.img.data();
  A.dest = plan.dest.data();
  std::vector<double> out(3 * (size_t)(nnz + nx), 0.0);
  if (s.setup_gpu) {
    int rc = near_eval_gpu(s, plan, out, err);
    if (rc) return rc;
  } else {
    parallel_for(Np, [&](int64_t b, int64_t e) {
      for (int64_t n = b; n < e; ++n) sm::near_eval_row(A, n, out.data());
    }, 64);
  }
  s.Ea.assign(out.begin(), out.begin() + 3 * nnz);
  for (auto& x : s.Ea) x *= s.Ms;
  s.Ex.rows = Np;
  s.Ex.comps = 3;
  s.Ex.rowptr.assign(Np + 1, 0);
  for (int64_t n = 0; n <= Np; ++n) s.Ex.rowptr[n] = (int32_t)plan.xptr[n];
  s.Ex.col = plan.xcol;
  s.Ex.vals.resize(3 * (size_t)nx);
  for (int64_t i = 0; i < 3 * nx; ++i) s.Ex.vals[i] = s.Ms * out[3 * nnz + i];
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
