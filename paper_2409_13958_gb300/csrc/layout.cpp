// Device layout of the unknowns (host side).  Unknowns are sorted by the grid box of their
// folded position, boxes ordered in tiles of TY rows x TZ planes with x fastest, so that
//   - the precorrection sources of an observer (all nodes in boxes within near_boxes) are
//     (2 nb + 1)^2 contiguous node ranges, one per neighbouring box row, and the matrix
//     needs no column indices: only its values are streamed;
//   - the projection of a tile's nodes lands in a small shared-memory region.
// Every operator is re-indexed to this order; user-facing arrays keep the unknown order
// of the C-ABI and are permuted at the boundary.
#include <algorithm>
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

int build_layout(const Setup& s, Layout& L, size_t smem_budget, size_t elem_bytes, Error& err) {
  const int64_t Np = s.Np;
  const int N[3] = {s.dims[0], s.dims[1], s.dims[2]};
  const int p = s.p, nb = s.near_boxes;
  L.pl = (p % 2 == 1) ? (p - 1) / 2 : p / 2;
  L.pr = (p % 2 == 1) ? (p + 1) / 2 : p / 2 + 1;
  // largest tile whose projection region fits the shared-memory budget
  L.tiled = false;
  L.TY = 1;
  L.TZ = 1;
  const int reach = L.pl + L.pr;
  for (int ty : {8, 4, 2, 1}) {
    for (int tz : {4, 2, 1}) {
      if (ty > N[1] || tz > N[2]) continue;
      size_t bytes = (size_t)(N[0] + reach) * (ty + reach) * (tz + reach) * elem_bytes;
      if (bytes <= smem_budget) {
        L.TY = ty;
        L.TZ = tz;
        L.tiled = true;
        break;
      }
    }
    if (L.tiled) break;
  }
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
  // SELL-32 copies
  const int64_t nch = (Np + 31) / 32;
  L.len.resize(Np);
  for (int64_t i = 0; i < Np; ++i) L.len[i] = L.rowptr[i + 1] - L.rowptr[i];
  L.sell_off.assign(nch + 1, 0);
  L.csell_off.assign(nch + 1, 0);
  for (int64_t c = 0; c < nch; ++c) {
    int64_t w = 0, wc = 0;
    for (int64_t i = 32 * c; i < std::min<int64_t>(Np, 32 * c + 32); ++i) {
      w = std::max<int64_t>(w, L.len[i]);
      wc = std::max<int64_t>(wc, L.cptr[i + 1] - L.cptr[i]);
    }
    L.sell_off[c + 1] = L.sell_off[c] + 32 * w;
    L.csell_off[c + 1] = L.csell_off[c] + 32 * wc;
  }
  const int64_t ns = L.sell_off[nch], ncs = L.csell_off[nch];
  L.col_s.assign(ns, 0);
  L.Wq_s.assign(3 * ns, 0.0);
  L.Ea_s.assign(3 * ns, 0.0);
  L.Gr_s.assign(3 * ns, 0.0);
  L.Kp_s.assign(ns, 0.0);
  L.cval_s.assign(ncs, 0.0);
  L.ccol_s.assign(ncs, 0);
  L.clen.resize(Np);
  for (int64_t i = 0; i < Np; ++i) L.clen[i] = (int32_t)(L.cptr[i + 1] - L.cptr[i]);
  parallel_for(nch, [&](int64_t b, int64_t e) {
    for (int64_t c = b; c < e; ++c) {
      const int64_t w = (L.sell_off[c + 1] - L.sell_off[c]) / 32;
      for (int64_t i = 32 * c; i < std::min<int64_t>(Np, 32 * c + 32); ++i) {
        const int64_t lane = i - 32 * c;
        for (int64_t j = 0; j < w; ++j) {
          const int64_t o = L.sell_off[c] + 32 * j + lane;
          if (j < L.len[i]) {
            const int64_t q = L.rowptr[i] + j;
            L.col_s[o] = L.col[q];
            L.Kp_s[o] = L.Kp[q];
            for (int d = 0; d < 3; ++d) {
              L.Wq_s[d * ns + o] = L.Wq[3 * q + d];
              L.Ea_s[d * ns + o] = L.Ea[3 * q + d];
              L.Gr_s[d * ns + o] = L.Gr[3 * q + d];
            }
          } else {
            L.col_s[o] = (int32_t)i;
          }
        }
        const int64_t cw = (L.csell_off[c + 1] - L.csell_off[c]) / 32;
        int64_t j = 0;
        for_segments(i, [&](int64_t k0, int64_t k1) {
          for (int64_t k = k0; k < k1; ++k, ++j) {
            L.cval_s[L.csell_off[c] + 32 * j + lane] = L.cval[L.cptr[i] + j];
            L.ccol_s[L.csell_off[c] + 32 * j + lane] = (int32_t)k;
          }
        });
        for (; j < cw; ++j) L.ccol_s[L.csell_off[c] + 32 * j + lane] = (int32_t)i;
      }
    }
  }, 256);

  // projection gather weights
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
  const int64_t G = (int64_t)N[0] * N[1] * N[2];
  const int64_t gch = (G + 31) / 32;
  std::vector<int32_t> glen(G);
  parallel_for(G, [&](int64_t b, int64_t e) {
    for (int64_t g = b; g < e; ++g) {
      int64_t n = 0;
      for_pull((int)(g % N[0]), (int)((g / N[0]) % N[1]), (int)(g / ((int64_t)N[0] * N[1])),
               [&](int64_t k0, int64_t k1) { n += k1 - k0; });
      glen[g] = (int32_t)n;
    }
  }, 4096);
  L.psell_off.assign(gch + 1, 0);
  for (int64_t c = 0; c < gch; ++c) {
    int64_t w = 0;
    for (int64_t g = 32 * c; g < std::min<int64_t>(G, 32 * c + 32); ++g) w = std::max<int64_t>(w, glen[g]);
    L.psell_off[c + 1] = L.psell_off[c] + 32 * w;
  }
  L.pw_s.assign(L.psell_off[gch], 0.0);
  L.pcol_s.assign(L.psell_off[gch], 0);
  L.plen = glen;
  parallel_for(G, [&](int64_t b, int64_t e) {
    for (int64_t g = b; g < e; ++g) {
      const int gc[3] = {(int)(g % N[0]), (int)((g / N[0]) % N[1]), (int)(g / ((int64_t)N[0] * N[1]))};
      int64_t o = L.psell_off[g / 32] + (g % 32);
      for_pull(gc[0], gc[1], gc[2], [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k, o += 32) {
          L.pcol_s[o] = (int32_t)k;
          if (!regular[k]) continue;
          double w = 1.0;
          for (int a = 0; a < 3; ++a) {
            int i = gc[a] - L.base[3 * k + a];
            if (s.periodic[a]) i = ((i % N[a]) + N[a]) % N[a];
            if (i < 0 || i > p) {
              w = 0.0;
              break;
            }
            w *= lagr(L.frac[3 * k + a], i);
          }
          L.pw_s[o] = w;
        }
      });
    }
  }, 4096);
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
