// Host set-up, part 3: the uniform grid (Eq. 16, read per axis), Lagrange stencils,
// the PGF spectrum used by BAIM step 2, and the point precorrection of step 4.
//   periodic axis:      Delta = L/N, origin = lowest folded coordinate, FFT length N
//   non-periodic axis:  m = ceil((p+1)/2) halo cells, Delta = D/(N-1-2m), FFT length 2N
//   stencil:            t = (x - origin)/Delta, base = floor(t) - (p-1)/2 (odd p) or
//                       round-half-down(t) - p/2 (even p), s = t - base
//   grid kernel:        K(d) = G^p(d Delta), K(0) = R(0)
//   precorrection:      C_nk += G0(r_n - r_k - l) - sum_a sum_b w_na w_kb G0'(r_a - r_b - l)
//                       for source images in boxes within near_boxes of the observer's box
#include <algorithm>
#include <cmath>

#include "internal.hpp"

namespace pmfem {

static inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static inline int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

int setup_grid(Setup& s, Error& err) {
  if (s.p < 2 || s.p > 5) {
    err = {EINVAL_, "order_p must be in 2..5"};
    return EINVAL_;
  }
  const int m = (s.p + 2) / 2;   // ceil((p+1)/2)
  for (int a = 0; a < 3; ++a) {
    double lo = 1e300, hi = -1e300;
    for (int64_t u = 0; u < s.Np; ++u) {
      lo = std::min(lo, s.pos_f[3 * u + a]);
      hi = std::max(hi, s.pos_f[3 * u + a]);
    }
    int N = s.dims_req[a];
    if (N <= 0) {   // about two grid points per mean edge length
      double span = s.periodic[a] ? s.L[a] : (hi - lo);
      N = (int)std::ceil(2.0 * span / s.mean_edge);
      if (!s.periodic[a]) N += 1 + 2 * m;
      N = std::max(N, s.periodic[a] ? std::max(2 * s.near_boxes + 2, s.p + 2) : 2 * m + 2);
      N = next_pow2(N);
      if (!s.periodic[a]) N = std::max(4, N);
      N = std::min(N, s.periodic[a] ? 1024 : 512);
    }
    s.dims[a] = N;
    if (s.periodic[a]) {
      if (N < 2 * s.near_boxes + 2 || N < s.p + 2) {
        err = {EINVAL_, "periodic grid axis needs N >= 2*near_boxes + 2 and N >= p + 2"};
        return EINVAL_;
      }
      s.delta[a] = s.L[a] / N;
      s.origin[a] = lo;
      s.fft[a] = N;
    } else {
      if (N < 2 * m + 2) {
        err = {EINVAL_, "non-periodic grid axis needs N >= 2*ceil((p+1)/2) + 2"};
        return EINVAL_;
      }
      if (!(hi > lo)) {
        err = {EMESH_, "mesh is flat along a non-periodic axis"};
        return EMESH_;
      }
      s.delta[a] = (hi - lo) / (N - 1 - 2 * m);
      s.origin[a] = lo - m * s.delta[a];
      s.fft[a] = 2 * N;
    }
    if (!is_pow2(s.fft[a]) || s.fft[a] < 4 || s.fft[a] > 1024) {
      err = {EINVAL_, "every FFT length must be a power of two in [4, 1024]"};
      return EINVAL_;
    }
  }
  s.base.assign(3 * s.Np, 0);
  s.frac.assign(3 * s.Np, 0.0);
  for (int64_t u = 0; u < s.Np; ++u)
    for (int a = 0; a < 3; ++a) {
      double t = (s.pos_f[3 * u + a] - s.origin[a]) / s.delta[a];
      int64_t b = (s.p % 2 == 1) ? (int64_t)std::floor(t) - (s.p - 1) / 2 : (int64_t)std::ceil(t - 0.5) - s.p / 2;
      if (!s.periodic[a] && (b < 0 || b + s.p > s.dims[a] - 1)) {
        err = {EINVAL_, "stencil leaves the grid"};
        return EINVAL_;
      }
      s.base[3 * u + a] = (int32_t)b;
      s.frac[3 * u + a] = t - (double)b;
    }
  return OK;
}

int setup_spectrum(Setup& s, Error& err) {
  if (s.setup_gpu) return spectrum_gpu(s, err);
  PeriodicGreen G(s.L);
  int U[3], K[3];
  for (int a = 0; a < 3; ++a) {
    U[a] = s.periodic[a] ? s.dims[a] / 2 + 1 : s.dims[a];   // distinct offsets |d|
    K[a] = s.fft[a] / 2 + 1;                                // distinct wavenumbers |k|
  }
  const int64_t nU = (int64_t)U[0] * U[1] * U[2];
  std::vector<double> Ku(nU);
  parallel_for(nU, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      int64_t dx = i % U[0], dy = (i / U[0]) % U[1], dz = i / ((int64_t)U[0] * U[1]);
      if (!dx && !dy && !dz) {
        Ku[i] = G.reg0();
      } else {
        Ku[i] = G(dx * s.delta[0], dy * s.delta[1], dz * s.delta[2]);
      }
    }
  }, 64);
  // even real kernel: FFT = separable cosine sums, sum_d c_d K(d) cos(2 pi d k / F),
  // c_d = 1 at d = 0 and at d = F/2, 2 otherwise
  std::vector<double> cur = Ku;
  int shape[3] = {U[0], U[1], U[2]};
  for (int a = 0; a < 3; ++a) {
    const int F = s.fft[a];
    std::vector<double> tab((size_t)K[a] * shape[a]);
    for (int k = 0; k < K[a]; ++k)
      for (int d = 0; d < shape[a]; ++d) {
        double c = (d == 0 || 2 * d == F) ? 1.0 : 2.0;
        tab[(size_t)k * shape[a] + d] = c * std::cos(2.0 * kPi * (double)(((int64_t)d * k) % F) / F);
      }
    int nshape[3] = {shape[0], shape[1], shape[2]};
    nshape[a] = K[a];
    const int64_t nout = (int64_t)nshape[0] * nshape[1] * nshape[2];
    std::vector<double> nxt(nout);
    const int64_t st_in[3] = {1, shape[0], (int64_t)shape[0] * shape[1]};
    parallel_for(nout, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        int64_t c[3] = {i % nshape[0], (i / nshape[0]) % nshape[1], i / ((int64_t)nshape[0] * nshape[1])};
        int64_t kk = c[a];
        c[a] = 0;
        int64_t off = c[0] * st_in[0] + c[1] * st_in[1] + c[2] * st_in[2];
        const double* row = &tab[(size_t)kk * shape[a]];
        double acc = 0;
        for (int d = 0; d < shape[a]; ++d) acc += row[d] * cur[off + d * st_in[a]];
        nxt[i] = acc;
      }
    }, 1024);
    cur.swap(nxt);
    shape[a] = K[a];
  }
  s.ghat.swap(cur);
  return OK;
}

using sm::lagrange;

int setup_precorrection(Setup& s, Error& err) {
  const int nb = s.near_boxes, p = s.p;
  const int64_t Np = s.Np;
  const int N0 = s.dims[0], N1 = s.dims[1], N2 = s.dims[2];
  // boxes and box -> unknown lists
  std::vector<int32_t> box(3 * Np);
  for (int64_t u = 0; u < Np; ++u)
    for (int a = 0; a < 3; ++a) {
      int64_t b = (int64_t)std::floor((s.pos_f[3 * u + a] - s.origin[a]) / s.delta[a]);
      b = std::max<int64_t>(0, std::min<int64_t>(b, s.dims[a] - 1));
      box[3 * u + a] = (int32_t)b;
    }
  s.box = box;
  const int64_t nbox = (int64_t)N0 * N1 * N2;
  std::vector<int64_t> bptr(nbox + 1, 0);
  auto lin = [&](int64_t x, int64_t y, int64_t z) { return x + (int64_t)N0 * (y + (int64_t)N1 * z); };
  for (int64_t u = 0; u < Np; ++u) bptr[lin(box[3 * u], box[3 * u + 1], box[3 * u + 2]) + 1]++;
  for (int64_t b = 0; b < nbox; ++b) bptr[b + 1] += bptr[b];
  std::vector<int32_t> bl(Np);
  {
    std::vector<int64_t> f(bptr.begin(), bptr.end() - 1);
    for (int64_t u = 0; u < Np; ++u) bl[f[lin(box[3 * u], box[3 * u + 1], box[3 * u + 2])]++] = (int32_t)u;
  }
  // table of G0' on integer grid offsets |d_a| <= R
  const int R = nb + p + 1, W = 2 * R + 1;
  std::vector<double> T0((size_t)W * W * W);
  for (int z = -R; z <= R; ++z)
    for (int y = -R; y <= R; ++y)
      for (int x = -R; x <= R; ++x) {
        double dx = x * s.delta[0], dy = y * s.delta[1], dz = z * s.delta[2];
        double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        T0[(size_t)(x + R) + W * ((size_t)(y + R) + W * (size_t)(z + R))] = (x || y || z) ? 1.0 / r : 0.0;
      }
  if (s.setup_gpu) return precorrection_gpu(s, box, bptr, bl, T0, R, err);
  std::vector<std::vector<std::pair<int32_t, double>>> rows(Np);
  const int dimN[3] = {N0, N1, N2};
  parallel_for(Np, [&](int64_t b, int64_t e) {
    std::vector<std::pair<int32_t, double>> acc;
    double wn[3][6];
    for (int64_t n = b; n < e; ++n) {
      acc.clear();
      for (int a = 0; a < 3; ++a) lagrange(s.frac[3 * n + a], p, wn[a]);
      const double* rn = &s.pos_f[3 * n];
      for (int oz = -nb; oz <= nb; ++oz)
        for (int oy = -nb; oy <= nb; ++oy)
          for (int ox = -nb; ox <= nb; ++ox) {
            int64_t t[3] = {box[3 * n] + ox, box[3 * n + 1] + oy, box[3 * n + 2] + oz};
            int64_t img[3] = {0, 0, 0};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
              if (s.periodic[a]) {
                int64_t q = t[a] >= 0 ? t[a] / dimN[a] : -((-t[a] + dimN[a] - 1) / dimN[a]);
                img[a] = q;
                t[a] -= q * dimN[a];
              } else if (t[a] < 0 || t[a] >= dimN[a]) {
                ok = false;
              }
            }
            if (!ok) continue;
            int64_t bi = lin(t[0], t[1], t[2]);
            for (int64_t q = bptr[bi]; q < bptr[bi + 1]; ++q) {
              const int32_t k = bl[q];
              int img3[3] = {(int)img[0], (int)img[1], (int)img[2]};
              int Db[3];
              for (int a = 0; a < 3; ++a) Db[a] = s.base[3 * n + a] - s.base[3 * (int64_t)k + a];
              const bool self = k == n && !img[0] && !img[1] && !img[2];
              const double v = sm::precorr_value(rn, &s.pos_f[3 * (int64_t)k], img3, s.L, Db, wn,
                                                 &s.frac[3 * (int64_t)k], p, dimN, T0.data(), R, self);
              acc.push_back({k, v});
            }
          }
      std::sort(acc.begin(), acc.end(), [](auto& x, auto& y) { return x.first < y.first; });
      std::vector<std::pair<int32_t, double>> merged;
      for (auto& x : acc) {
        if (!merged.empty() && merged.back().first == x.first) merged.back().second += x.second;
        else merged.push_back(x);
      }
      rows[n].swap(merged);
    }
  }, 64);
  s.C.rows = Np;
  s.C.comps = 1;
  s.C.rowptr.assign(Np + 1, 0);
  for (int64_t n = 0; n < Np; ++n) s.C.rowptr[n + 1] = s.C.rowptr[n] + (int32_t)rows[n].size();
  s.C.col.resize(s.C.rowptr[Np]);
  s.C.vals.resize(s.C.rowptr[Np]);
  for (int64_t n = 0; n < Np; ++n) {
    int64_t o = s.C.rowptr[n];
    for (size_t i = 0; i < rows[n].size(); ++i) {
      s.C.col[o + i] = rows[n][i].first;
      s.C.vals[o + i] = rows[n][i].second;
    }
  }
  return OK;
}

}  // namespace pmfem
