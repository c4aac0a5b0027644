// Host set-up, part 2: periodized P1 operators assembled element by element with
// vertex indices mapped to their unknowns (cases 1-3 of Sec. 3.1 and the de-duplication
// of Eq. 11 follow from visiting every tetrahedron once), on one adjacency pattern
// shared by the exchange (Eq. 8), charge (Eq. 14a) and gradient (Eq. 14d) operators.
#include <algorithm>
#include <cmath>

#include "internal.hpp"

namespace pmfem {

static void load_tet(const Setup& s, int64_t e, double X[4][3]) {
  for (int i = 0; i < 4; ++i) {
    int32_t v = s.tets[4 * e + i];
    for (int d = 0; d < 3; ++d) X[i][d] = s.xyz[3 * (int64_t)v + d];
  }
}

int setup_operators(Setup& s, Error& err) {
  const int64_t Np = s.Np, T = s.T;
  // incidence: unknown -> (tet, local vertex) slots
  std::vector<int64_t> inc_ptr(Np + 1, 0);
  for (int64_t i = 0; i < 4 * T; ++i) inc_ptr[s.lca[s.tets[i]] + 1]++;
  for (int64_t u = 0; u < Np; ++u) inc_ptr[u + 1] += inc_ptr[u];
  std::vector<int64_t> inc(4 * T), fill(inc_ptr.begin(), inc_ptr.end() - 1);
  for (int64_t i = 0; i < 4 * T; ++i) inc[fill[s.lca[s.tets[i]]]++] = i;

  // adjacency pattern: unknowns sharing a tetrahedron (after mapping), sorted per row
  std::vector<int32_t> cnt(Np + 1, 0);
  std::vector<std::vector<int32_t>> rows(Np);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    std::vector<int32_t> buf;
    for (int64_t u = b; u < e; ++u) {
      buf.clear();
      for (int64_t t = inc_ptr[u]; t < inc_ptr[u + 1]; ++t) {
        int64_t tet = inc[t] / 4;
        for (int j = 0; j < 4; ++j) buf.push_back(s.lca[s.tets[4 * tet + j]]);
      }
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
      rows[u] = buf;
    }
  });
  s.rowptr.assign(Np + 1, 0);
  for (int64_t u = 0; u < Np; ++u) s.rowptr[u + 1] = s.rowptr[u] + (int32_t)rows[u].size();
  const int64_t nnz = s.rowptr[Np];
  if (nnz > 2000000000LL) {
    err = {EINVAL_, "adjacency has more than 2e9 entries"};
    return EINVAL_;
  }
  s.col.resize(nnz);
  for (int64_t u = 0; u < Np; ++u) std::copy(rows[u].begin(), rows[u].end(), s.col.begin() + s.rowptr[u]);
  rows.clear();
  rows.shrink_to_fit();

  std::vector<double> K(nnz, 0.0), W(3 * nnz, 0.0);
  s.V.assign(Np, 0.0);
  auto find = [&](int64_t row, int32_t c) -> int64_t {
    const int32_t* b = s.col.data() + s.rowptr[row];
    const int32_t* e = s.col.data() + s.rowptr[row + 1];
    const int32_t* p = std::lower_bound(b, e, c);
    return (int64_t)(p - s.col.data());
  };
  parallel_for(Np, [&](int64_t b, int64_t e) {
    for (int64_t u = b; u < e; ++u) {
      for (int64_t t = inc_ptr[u]; t < inc_ptr[u + 1]; ++t) {
        int64_t tet = inc[t] / 4;
        int i = (int)(inc[t] % 4);
        double X[4][3], g[4][3];
        load_tet(s, tet, X);
        double Ve = tet_grads(X, g);
        s.V[u] += 0.25 * Ve;
        const double Ke = s.A_tet.empty() ? Ve : s.A_tet[tet] * Ve;   // stiffness inside the element sum
        for (int j = 0; j < 4; ++j) {
          int64_t pos = find(u, s.lca[s.tets[4 * tet + j]]);
          K[pos] += Ke * (g[i][0] * g[j][0] + g[i][1] * g[j][1] + g[i][2] * g[j][2]);
          for (int d = 0; d < 3; ++d) W[3 * pos + d] += 0.25 * Ve * g[i][d];
        }
      }
    }
  });
  // scaled values used by the field kernels
  // H_ex = -(2 A/(mu0 Ms)) V^-1 K m; with a stiffness per tetrahedron A sits inside K
  const double cex = s.A_tet.empty() ? -2.0 * s.A / (kMu0 * s.Ms) : -2.0 / (kMu0 * s.Ms);
  s.Kp.resize(nnz);
  s.Wq.resize(3 * nnz);
  s.Gr.resize(3 * nnz);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    for (int64_t u = b; u < e; ++u)
      for (int64_t p = s.rowptr[u]; p < s.rowptr[u + 1]; ++p) {
        s.Kp[p] = cex * K[p] / s.V[u];
        int32_t k = s.col[p];
        int64_t q = find(k, (int32_t)u);   // (W^q)_{k u}: transpose entry
        for (int d = 0; d < 3; ++d) {
          s.Wq[3 * p + d] = s.Ms * W[3 * p + d];
          s.Gr[3 * p + d] = -W[3 * q + d] / (4.0 * kPi * s.V[u]);
        }
      }
  });

  // true boundary faces: mapped vertex triples that occur once.  Faces are bucketed by their
  // smallest unknown (a counting sort), each bucket sorted on its own: the same order as one
  // global sort by (a, b, c, ref), in parallel.
  struct F {
    int32_t a, b, c;
    int64_t ref;
  };
  static const int opp[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
  std::vector<int64_t> fptr(Np + 1, 0);
  auto face_key = [&](int64_t slot, int32_t m[3]) {
    const int64_t t = slot / 4;
    const int f = (int)(slot % 4);
    for (int j = 0; j < 3; ++j) m[j] = s.lca[s.tets[4 * t + opp[f][j]]];
    std::sort(m, m + 3);
  };
  for (int64_t i = 0; i < 4 * T; ++i) {
    int32_t m[3];
    face_key(i, m);
    fptr[m[0] + 1]++;
  }
  for (int64_t u = 0; u < Np; ++u) fptr[u + 1] += fptr[u];
  std::vector<F> faces(4 * T);
  {
    std::vector<int64_t> fill(fptr.begin(), fptr.end() - 1);
    for (int64_t i = 0; i < 4 * T; ++i) {
      int32_t m[3];
      face_key(i, m);
      faces[fill[m[0]]++] = {m[0], m[1], m[2], i};
    }
  }
  std::vector<std::vector<int32_t>> bf_rows(Np);
  parallel_for(Np, [&](int64_t ub, int64_t ue) {
    for (int64_t u = ub; u < ue; ++u) {
      std::sort(faces.begin() + fptr[u], faces.begin() + fptr[u + 1], [](const F& x, const F& y) {
        if (x.b != y.b) return x.b < y.b;
        if (x.c != y.c) return x.c < y.c;
        return x.ref < y.ref;
      });
      for (int64_t i = fptr[u]; i < fptr[u + 1];) {
        int64_t j = i + 1;
        while (j < fptr[u + 1] && faces[j].b == faces[i].b && faces[j].c == faces[i].c) ++j;
        if (j - i == 1) {
          const int64_t t = faces[i].ref / 4;
          const int f = (int)(faces[i].ref % 4);
          int32_t v[3];
          for (int k = 0; k < 3; ++k) v[k] = s.tets[4 * t + opp[f][k]];
          // outward with respect to the owning tetrahedron
          double X[4][3];
          load_tet(s, t, X);
          double cen[3] = {0, 0, 0};
          for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) cen[d] += 0.25 * X[k][d];
          const double* pa = &s.xyz[3 * (int64_t)v[0]];
          const double* pb = &s.xyz[3 * (int64_t)v[1]];
          const double* pc = &s.xyz[3 * (int64_t)v[2]];
          double e1[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
          double e2[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
          double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
          double out = n[0] * (pa[0] - cen[0]) + n[1] * (pa[1] - cen[1]) + n[2] * (pa[2] - cen[2]);
          if (out < 0) std::swap(v[1], v[2]);
          bf_rows[u].insert(bf_rows[u].end(), v, v + 3);
        }
        i = j;
      }
    }
  }, 1024);
  s.bfaces.clear();
  for (int64_t u = 0; u < Np; ++u) s.bfaces.insert(s.bfaces.end(), bf_rows[u].begin(), bf_rows[u].end());
  std::vector<F>().swap(faces);

  // mean length of the unique edges of the original mesh: edges bucketed by their smaller
  // node, each bucket sorted and de-duplicated in parallel, lengths summed per bucket and the
  // bucket sums added in node order
  static const int ep[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  const int64_t N = s.N;
  std::vector<int64_t> eptr(N + 1, 0);
  for (int64_t t = 0; t < T; ++t)
    for (int k = 0; k < 6; ++k) {
      const int32_t a0 = s.tets[4 * t + ep[k][0]], b0 = s.tets[4 * t + ep[k][1]];
      eptr[std::min(a0, b0) + 1]++;
    }
  for (int64_t u = 0; u < N; ++u) eptr[u + 1] += eptr[u];
  std::vector<int32_t> other(eptr[N]);
  {
    std::vector<int64_t> fill(eptr.begin(), eptr.end() - 1);
    for (int64_t t = 0; t < T; ++t)
      for (int k = 0; k < 6; ++k) {
        const int32_t a0 = s.tets[4 * t + ep[k][0]], b0 = s.tets[4 * t + ep[k][1]];
        other[fill[std::min(a0, b0)]++] = std::max(a0, b0);
      }
  }
  std::vector<double> bucket_len(N, 0.0);
  std::vector<int64_t> bucket_cnt(N, 0);
  parallel_for(N, [&](int64_t ub, int64_t ue) {
    for (int64_t a = ub; a < ue; ++a) {
      auto b0 = other.begin() + eptr[a], b1 = other.begin() + eptr[a + 1];
      std::sort(b0, b1);
      b1 = std::unique(b0, b1);
      bucket_cnt[a] = b1 - b0;
      double acc = 0;
      for (auto it = b0; it != b1; ++it) {
        const int64_t b = *it;
        double d0 = s.xyz[3 * a] - s.xyz[3 * b], d1 = s.xyz[3 * a + 1] - s.xyz[3 * b + 1],
               d2 = s.xyz[3 * a + 2] - s.xyz[3 * b + 2];
        acc += std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      }
      bucket_len[a] = acc;
    }
  }, 1024);
  double acc = 0;
  int64_t ne = 0;
  for (int64_t a = 0; a < N; ++a) {
    acc += bucket_len[a];
    ne += bucket_cnt[a];
  }
  s.mean_edge = acc / (double)ne;
  return OK;
}

}  // namespace pmfem
