// Device layout of the unknowns (host side).  Unknowns are sorted by the grid box of their
// folded position (z-major, then y, x fastest), so that the sources of every sparse row lie
// at nearby indices: the precorrection sources of an observer (all nodes in boxes within
// near_boxes) are (2 nb + 1)^2 contiguous node ranges, and the nodes feeding a grid point
// in the projection are (p + 1)^2 such ranges.  Every operator is re-indexed to this
// order and stored in SELL-32 with column deltas (16-bit when they fit); user-facing
// arrays keep the unknown order of the C-ABI and are permuted at the boundary.
#include <algorithm>
#include <functional>
#include <numeric>

#include "internal.hpp"

namespace pmfem {

namespace {
// x-segments of one neighbouring box row, in enumeration order (shared with the kernel)
int x_segments(int bx, int nb, int N0, bool per, int lo_out[2], int hi_out[2]) {
  int lo = bx - nb, hi = bx + nb;
  if (!per) {
    lo = std::max(lo, 0);
    hi = std::min(hi, N0 - 1);
    if (lo > hi) return 0;
    lo_out[0] = lo;
    hi_out[0] = hi;
    return 1;
  }
  if (lo < 0) {
    lo_out[0] = lo + N0, hi_out[0] = N0 - 1;
    lo_out[1] = 0, hi_out[1] = hi;
    return 2;
  }
  if (hi >= N0) {
    lo_out[0] = lo, hi_out[0] = N0 - 1;
    lo_out[1] = 0, hi_out[1] = hi - N0;
    return 2;
  }
  lo_out[0] = lo;
  hi_out[0] = hi;
  return 1;
}

bool wrap_axis(int& v, int N, bool per) {
  if (per) {
    if (v < 0) v += N;
    if (v >= N) v -= N;
    return true;
  }
  return v >= 0 && v < N;
}
}  // namespace

// SELL-32 from row callbacks: len(r), base(r) and fill(r, put(col, values[comps])).  With
// sigma > 1, rows are sorted by decreasing length inside windows of sigma rows so that
// the 32 rows of a chunk have similar lengths (little padding).
//
// Columns are stored as deltas modulo ncols to a per-row base: a column c is recovered as
// (base + delta) wrapped into [0, ncols).  The base is moved from base(r) to the middle of
// the row's columns (measured modulo ncols), so that rows whose sources straddle the
// periodic seam of the box order (the last and the first boxes along a periodic axis) still
// have small deltas.
int64_t centre_deltas(const int32_t* cols, int64_t len, int32_t ref, int64_t n, int32_t* base, int32_t* delta) {
  const int64_t nc = std::max<int64_t>(n, 1);
  const int64_t half = nc / 2;
  auto modd = [&](int64_t d) {   // d modulo nc, in [-(nc - nc/2) + 1, nc/2]
    d %= nc;
    if (d < 0) d += nc;
    return d > half ? d - nc : d;
  };
  int64_t lo = 0, hi = 0;
  for (int64_t k = 0; k < len; ++k) {
    const int64_t d = modd((int64_t)cols[k] - ref);
    lo = k ? std::min(lo, d) : d;
    hi = k ? std::max(hi, d) : d;
  }
  int64_t b = ref + (lo + hi) / 2;
  b = ((b % nc) + nc) % nc;
  *base = (int32_t)b;
  int64_t md = 0;
  for (int64_t k = 0; k < len; ++k) {
    const int64_t d = modd((int64_t)cols[k] - b);
    md = std::max<int64_t>(md, d < 0 ? -d : d);
    delta[k] = (int32_t)d;
  }
  return md;
}

void build_sell(SellMatrix& M, int64_t rows, int comps, int sigma, int col_bits, int64_t ncols, int vw,
                const std::function<int64_t(int64_t)>& len,
                const std::function<int32_t(int64_t)>& base,
                const std::function<void(int64_t, const std::function<void(int32_t, const double*)>&)>& fill,
                bool drop_empty = false) {
  M.comps = comps;
  M.vw = vw;
  std::vector<int64_t> rl(rows);
  parallel_for(rows, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) rl[r] = len(r);
  }, 4096);
  M.map.resize(rows);
  std::iota(M.map.begin(), M.map.end(), 0);
  if (sigma > 1)
    for (int64_t w0 = 0; w0 < rows; w0 += sigma) {
      const int64_t w1 = std::min(rows, w0 + sigma);
      std::stable_sort(M.map.begin() + w0, M.map.begin() + w1, [&](int32_t a, int32_t b) { return rl[a] > rl[b]; });
    }
  // drop_empty: when at least half of the rows have no entries, they are left out (the caller
  // zeroes their results); otherwise every row stays (and writes its zero itself)
  int64_t nempty = 0;
  if (drop_empty)
    for (int64_t r = 0; r < rows; ++r) nempty += rl[r] == 0;
  if (drop_empty && 2 * nempty >= rows && nempty > 0) {
    int64_t k = 0;
    for (int64_t t = 0; t < rows; ++t)
      if (rl[M.map[t]] > 0) M.map[k++] = M.map[t];
    M.map.resize(k);
    rows = k;
  }
  M.rows = rows;
  const int64_t nch = (rows + 31) / 32;
  M.len.resize(rows);
  M.base.resize(rows);
  M.off.assign(nch + 1, 0);
  for (int64_t t = 0; t < rows; ++t) M.len[t] = (int32_t)rl[M.map[t]];
  for (int64_t c = 0; c < nch; ++c) {
    int64_t w = 0;
    for (int64_t t = 32 * c; t < std::min(rows, 32 * c + 32); ++t) w = std::max<int64_t>(w, M.len[t]);
    w = (w + vw - 1) / vw * vw;   // whole vectors per lane
    M.off[c + 1] = M.off[c] + 32 * w;
  }
  const int64_t P = M.off[nch];
  std::vector<int32_t> delta(P, 0);
  M.val.assign((size_t)comps * P, 0.0);
  int64_t maxd = 0;
  std::vector<int64_t> maxd_t(nch, 0);
  parallel_for(nch, [&](int64_t cb, int64_t ce) {
    std::vector<int32_t> cols;
    std::vector<double> vals;
    for (int64_t c = cb; c < ce; ++c) {
      int64_t md = 0;
      for (int64_t t = 32 * c; t < std::min(rows, 32 * c + 32); ++t) {
        const int64_t r = M.map[t];
        const int32_t ref = base(r);
        cols.clear();
        vals.clear();
        fill(r, [&](int32_t col, const double* v) {
          cols.push_back(col);
          vals.insert(vals.end(), v, v + comps);
        });
        int32_t bse;
        std::vector<int32_t> d(cols.size());
        md = std::max(md, centre_deltas(cols.data(), (int64_t)cols.size(), ref, ncols, &bse, d.data()));
        M.base[t] = bse;
        const int64_t lane = t - 32 * c;
        for (size_t k = 0; k < cols.size(); ++k) {
          const int64_t o = M.off[c] + ((int64_t)(k / vw) * 32 + lane) * vw + (int64_t)(k % vw);
          delta[o] = d[k];
          for (int q = 0; q < comps; ++q) M.val[(size_t)q * P + o] = vals[k * comps + q];
        }
      }
      maxd_t[c] = md;
    }
  }, 64);
  for (int64_t c = 0; c < nch; ++c) maxd = std::max(maxd, maxd_t[c]);
  M.col16 = col_bits == 16 ? maxd <= 32767 : (col_bits == 32 ? false : maxd <= 32767);
  if (M.col16) {
    M.d16.assign(delta.begin(), delta.end());
    M.d32.clear();
  } else {
    M.d32.swap(delta);
    M.d16.clear();
  }
}

int build_layout(const Setup& s, Layout& L, Error& err) {
  const int64_t Np = s.Np;
  const int N[3] = {s.dims[0], s.dims[1], s.dims[2]};
  const int p = s.p, nb = s.near_boxes;
  L.pl = (p % 2 == 1) ? (p - 1) / 2 : p / 2;
  L.pr = (p % 2 == 1) ? (p + 1) / 2 : p / 2 + 1;
  // box order: tiles of TY rows x TZ planes (defaults favour gather locality)
  L.TY = s.tile_y > 0 ? s.tile_y : 8;
  L.TZ = s.tile_z > 0 ? s.tile_z : 4;
  while (L.TY > 1 && N[1] % L.TY) L.TY /= 2;
  while (L.TZ > 1 && N[2] % L.TZ) L.TZ /= 2;
  L.TY = std::min(L.TY, N[1]);
  L.TZ = std::min(L.TZ, N[2]);
  // permutation: by box index, then by unknown index
  std::vector<int64_t> key(Np);
  for (int64_t u = 0; u < Np; ++u) key[u] = L.box_index(s.box[3 * u], s.box[3 * u + 1], s.box[3 * u + 2], N);
  L.perm.resize(Np);
  std::iota(L.perm.begin(), L.perm.end(), 0);
  std::stable_sort(L.perm.begin(), L.perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::vector<int32_t> iperm(Np);
  for (int64_t i = 0; i < Np; ++i) iperm[L.perm[i]] = (int32_t)i;
  const int64_t nbox = (int64_t)N[0] * N[1] * N[2];
  L.bstart.assign(nbox + 1, 0);
  for (int64_t u = 0; u < Np; ++u) L.bstart[key[u] + 1]++;
  for (int64_t b = 0; b < nbox; ++b) L.bstart[b + 1] += L.bstart[b];
  L.box.resize(3 * Np);
  L.base.resize(3 * Np);
  L.frac.resize(3 * Np);
  for (int64_t i = 0; i < Np; ++i)
    for (int a = 0; a < 3; ++a) {
      const int64_t u = L.perm[i];
      L.box[3 * i + a] = s.box[3 * u + a];
      L.base[3 * i + a] = s.base[3 * u + a];
      L.frac[3 * i + a] = s.frac[3 * u + a];
    }
  // adjacency and its values, rows and columns re-indexed, columns sorted
  const int64_t nnz = (int64_t)s.col.size();
  L.rowptr.assign(Np + 1, 0);
  for (int64_t i = 0; i < Np; ++i) {
    const int64_t u = L.perm[i];
    L.rowptr[i + 1] = L.rowptr[i] + (s.rowptr[u + 1] - s.rowptr[u]);
  }
  L.col.resize(nnz);
  L.Wq.resize(3 * nnz);
  L.Ea.resize(3 * nnz);
  L.Gr.resize(3 * nnz);
  L.Kp.resize(nnz);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    std::vector<std::pair<int32_t, int64_t>> ent;
    for (int64_t i = b; i < e; ++i) {
      const int64_t u = L.perm[i];
      ent.clear();
      for (int64_t q = s.rowptr[u]; q < s.rowptr[u + 1]; ++q) ent.push_back({iperm[s.col[q]], q});
      std::sort(ent.begin(), ent.end());
      int64_t o = L.rowptr[i];
      for (auto& x : ent) {
        L.col[o] = x.first;
        L.Kp[o] = s.Kp[x.second];
        for (int d = 0; d < 3; ++d) {
          L.Wq[3 * o + d] = s.Wq[3 * x.second + d];
          L.Ea[3 * o + d] = s.Ea[3 * x.second + d];
          L.Gr[3 * o + d] = s.Gr[3 * x.second + d];
        }
        ++o;
      }
    }
  });
  // near-element entries beyond the pattern
  L.Ex.rows = Np;
  L.Ex.comps = 3;
  L.Ex.rowptr.assign(Np + 1, 0);
  for (int64_t i = 0; i < Np; ++i) {
    const int64_t u = L.perm[i];
    L.Ex.rowptr[i + 1] = L.Ex.rowptr[i] + (s.Ex.rowptr[u + 1] - s.Ex.rowptr[u]);
  }
  L.Ex.col.resize(s.Ex.col.size());
  L.Ex.vals.resize(s.Ex.vals.size());
  for (int64_t i = 0; i < Np; ++i) {
    const int64_t u = L.perm[i];
    int64_t o = L.Ex.rowptr[i];
    for (int64_t q = s.Ex.rowptr[u]; q < s.Ex.rowptr[u + 1]; ++q, ++o) {
      L.Ex.col[o] = iperm[s.Ex.col[q]];
      for (int d = 0; d < 3; ++d) L.Ex.vals[3 * o + d] = s.Ex.vals[3 * q + d];
    }
  }
  // precorrection values in segment order
  auto for_segments = [&](int64_t i, auto&& fn) {
    const int bx = L.box[3 * i], by = L.box[3 * i + 1], bz = L.box[3 * i + 2];
    for (int dz = -nb; dz <= nb; ++dz) {
      int z = bz + dz;
      if (!wrap_axis(z, N[2], s.periodic[2])) continue;
      for (int dy = -nb; dy <= nb; ++dy) {
        int y = by + dy;
        if (!wrap_axis(y, N[1], s.periodic[1])) continue;
        int lo[2], hi[2];
        const int ns = x_segments(bx, nb, N[0], s.periodic[0], lo, hi);
        for (int g = 0; g < ns; ++g) {
          const int64_t k0 = L.bstart[L.box_index(lo[g], y, z, N)];
          const int64_t k1 = L.bstart[L.box_index(hi[g], y, z, N) + 1];
          fn(k0, k1);
        }
      }
    }
  };
  L.cptr.assign(Np + 1, 0);
  for (int64_t i = 0; i < Np; ++i) {
    int64_t len = 0;
    for_segments(i, [&](int64_t k0, int64_t k1) { len += k1 - k0; });
    L.cptr[i + 1] = L.cptr[i] + len;
  }
  L.cval.assign(L.cptr[Np], 0.0);
  L.ccol.assign(L.cptr[Np], 0);
  std::vector<char> bad(Np, 0);
  parallel_for(Np, [&](int64_t b, int64_t e) {
    std::vector<char> used;
    for (int64_t i = b; i < e; ++i) {
      const int64_t u = L.perm[i];
      const int32_t* cb = s.C.col.data() + s.C.rowptr[u];
      const int64_t rl = s.C.rowptr[u + 1] - s.C.rowptr[u];
      used.assign(rl, 0);
      int64_t o = L.cptr[i], consumed = 0;
      for_segments(i, [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k, ++o) {
          L.ccol[o] = (int32_t)k;
          const int32_t ku = L.perm[k];
          const int32_t* it = std::lower_bound(cb, cb + rl, ku);
          const int64_t pos = it - cb;
          if (pos < rl && *it == ku && !used[pos]) {
            used[pos] = 1;
            L.cval[o] = s.C.vals[s.C.rowptr[u] + pos];
            ++consumed;
          }
        }
      });
      if (consumed != rl) bad[i] = 1;
    }
  }, 64);
  for (int64_t i = 0; i < Np; ++i)
    if (bad[i]) {
      err = {EINVAL_, "precorrection layout does not cover row " + std::to_string(i)};
      return EINVAL_;
    }
  // SELL-32 operators
  build_sell(L.adj, Np, 10, 1, s.col_bits, Np, 4, [&](int64_t i) { return (int64_t)(L.rowptr[i + 1] - L.rowptr[i]); },
             [&](int64_t i) { return (int32_t)i; },
             [&](int64_t i, const std::function<void(int32_t, const double*)>& put) {
               for (int64_t q = L.rowptr[i]; q < L.rowptr[i + 1]; ++q) {
                 const double v[10] = {L.Wq[3 * q], L.Wq[3 * q + 1], L.Wq[3 * q + 2], L.Ea[3 * q], L.Ea[3 * q + 1],
                                       L.Ea[3 * q + 2], L.Gr[3 * q], L.Gr[3 * q + 1], L.Gr[3 * q + 2], L.Kp[q]};
                 put(L.col[q], v);
               }
             });
  // rows sorted by length in windows of 1024 (about a dozen box rows): a warp's rows stay
  // near one another (shared gathers) and have similar lengths (little idle lanes)
  build_sell(L.cor, Np, 1, s.sort_window > 0 ? s.sort_window : 1024, s.col_bits, Np, PMFEM_COR_VW,
               [&](int64_t i) { return L.cptr[i + 1] - L.cptr[i]; }, [&](int64_t i) { return (int32_t)i; },
               [&](int64_t i, const std::function<void(int32_t, const double*)>& put) {
                 for (int64_t o = L.cptr[i]; o < L.cptr[i + 1]; ++o) put(L.ccol[o], &L.cval[o]);
               });

  // projection P^T: grid point g gathers from the nodes whose stencil covers it
  auto lagr = [&](double sv, int i) {
    double v = 1.0;
    for (int j = 0; j <= p; ++j)
      if (j != i) v *= (sv - j) / (double)(i - j);
    return v;
  };
  std::vector<char> regular(Np, 1);
  for (int64_t i = 0; i < Np; ++i)
    for (int a = 0; a < 3; ++a) {
      const int d = L.base[3 * i + a] - (L.box[3 * i + a] - L.pl);
      if (!(d == 0 || (p % 2 == 0 && d == 1))) regular[i] = 0;
    }
  auto for_pull = [&](int gx, int gy, int gz, auto&& fn) {
    for (int bz = gz - L.pr; bz <= gz + L.pl; ++bz) {
      int z = bz;
      if (!wrap_axis(z, N[2], s.periodic[2])) continue;
      for (int by = gy - L.pr; by <= gy + L.pl; ++by) {
        int y = by;
        if (!wrap_axis(y, N[1], s.periodic[1])) continue;
        int lo = gx - L.pr, hi = gx + L.pl, lo2 = 0, hi2 = -1;
        if (!s.periodic[0]) {
          lo = std::max(lo, 0);
          hi = std::min(hi, N[0] - 1);
        } else if (lo < 0) {
          lo2 = 0, hi2 = hi, lo = lo + N[0], hi = N[0] - 1;
        } else if (hi >= N[0]) {
          lo2 = 0, hi2 = hi - N[0], hi = N[0] - 1;
        }
        if (lo <= hi) fn(L.bstart[L.box_index(lo, y, z, N)], L.bstart[L.box_index(hi, y, z, N) + 1]);
        if (lo2 <= hi2) fn(L.bstart[L.box_index(lo2, y, z, N)], L.bstart[L.box_index(hi2, y, z, N) + 1]);
      }
    }
  };
  auto gcoord = [&](int64_t g, int gc[3]) {
    gc[0] = (int)(g % N[0]);
    gc[1] = (int)((g / N[0]) % N[1]);
    gc[2] = (int)(g / ((int64_t)N[0] * N[1]));
  };
  const int64_t G = (int64_t)N[0] * N[1] * N[2];
  // the grid points no node projects to (the padding of open axes, the space around the body) are
  // left out of the projection's rows when they are at least half of the grid (thin films): the
  // grid is then cleared before each projection instead
  build_sell(L.pro, G, 1, s.sort_window > 0 ? s.sort_window : 1024, s.col_bits, Np, PMFEM_COR_VW,
             [&](int64_t g) {
               int gc[3];
               gcoord(g, gc);
               int64_t n = 0;
               for_pull(gc[0], gc[1], gc[2], [&](int64_t k0, int64_t k1) { n += k1 - k0; });
               return n;
             },
             [&](int64_t g) {
               int gc[3];
               gcoord(g, gc);
               return L.bstart[L.box_index(gc[0], gc[1], gc[2], N)];
             },
             [&](int64_t g, const std::function<void(int32_t, const double*)>& put) {
               int gc[3];
               gcoord(g, gc);
               for_pull(gc[0], gc[1], gc[2], [&](int64_t k0, int64_t k1) {
                 for (int64_t k = k0; k < k1; ++k) {
                   double w = regular[k] ? 1.0 : 0.0;
                   for (int a = 0; a < 3 && w != 0.0; ++a) {
                     int i = gc[a] - L.base[3 * k + a];
                     if (s.periodic[a]) i = ((i % N[a]) + N[a]) % N[a];
                     w = (i < 0 || i > p) ? 0.0 : w * lagr(L.frac[3 * k + a], i);
                   }
                   put((int32_t)k, &w);
                 }
               });
             },
             true);
  L.xnode.clear();
  L.xgrid.clear();
  L.xw.clear();
  for (int64_t k = 0; k < Np; ++k) {
    if (regular[k]) continue;
    for (int c = 0; c <= p; ++c)
      for (int bj = 0; bj <= p; ++bj)
        for (int ai = 0; ai <= p; ++ai) {
          int gi[3] = {L.base[3 * k] + ai, L.base[3 * k + 1] + bj, L.base[3 * k + 2] + c};
          for (int a = 0; a < 3; ++a)
            if (s.periodic[a]) gi[a] = ((gi[a] % N[a]) + N[a]) % N[a];
          L.xnode.push_back((int32_t)k);
          L.xgrid.push_back(gi[0] + (int64_t)N[0] * (gi[1] + (int64_t)N[1] * gi[2]));
          L.xw.push_back(lagr(L.frac[3 * k], ai) * lagr(L.frac[3 * k + 1], bj) * lagr(L.frac[3 * k + 2], c));
        }
  }
  return OK;
}

}  // namespace pmfem
