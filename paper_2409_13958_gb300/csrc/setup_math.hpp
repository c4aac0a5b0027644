// Set-up arithmetic shared by the host set-up (g++) and the GPU set-up (nvcc): the
// periodic Green's function of Eq. 15 (k0 = 0, Ewald-type splitting), the exact potential
// integrals of the near-element correction (Sec. 3.2, Eq. 14c), the Lagrange weights of the
// stencils (Eq. 16 grid) and the P1 gradients.  Every function is written once and compiled
// for both sides, so the two set-up paths evaluate the same formulas in the same order (they
// differ only by the last-bit rounding of the host's and the device's libm).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define PMFEM_HD __host__ __device__ __forceinline__
#else
#define PMFEM_HD inline
#endif

namespace pmfem {
namespace sm {

constexpr double kPiD = 3.14159265358979323846;
constexpr double kCutReal = 6.3;   // erfc(6.3) ~ 1e-19
constexpr double kCutSpec = 43.0;  // exp(-43) ~ 2e-19
constexpr double kEulerGamma = 0.57721566490153286061;
constexpr int kGaussLegendre = 48;

PMFEM_HD void sub(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
PMFEM_HD double dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
PMFEM_HD void cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// ------------------------------------------------------------------ P1 tetrahedron
// Signed volume and the gradients of the four barycentric coordinates.
PMFEM_HD double tet_grads(const double X[4][3], double g[4][3]) {
  double e1[3], e2[3], e3[3], c23[3], c31[3], c12[3];
  sub(X[1], X[0], e1);
  sub(X[2], X[0], e2);
  sub(X[3], X[0], e3);
  cross(e2, e3, c23);
  cross(e3, e1, c31);
  cross(e1, e2, c12);
  const double det = dot(e1, c23);
  for (int d = 0; d < 3; ++d) {
    g[1][d] = c23[d] / det;
    g[2][d] = c31[d] / det;
    g[3][d] = c12[d] / det;
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  return det / 6.0;
}

// ------------------------------------------------------------------ exact integrals
// Triangle (unit normal n, observer r, its projection p on the plane, height d): with every
// edge taken counter-clockwise about n from P- to P+, direction l, in-plane outward normal
// u = l x n, t = (P- - p).u, l+- = (P+- - p).l, R0^2 = t^2 + d^2, R+- = |P+- - r| and
// f = ln((R+ + l+)/(R- + l-)), integrating 1/R in polar form about p edge by edge gives
//   int dS/R        = sum [t f - |d| (atan(t l+/(R0^2+|d|R+)) - atan(t l-/(R0^2+|d|R-)))]
//   int (r'-p)/R dS = 1/2 sum u [R0^2 f + l+ R+ - l- R-]
// (the published closed forms of Wilton et al., IEEE TAP 32(3), 1984).
PMFEM_HD void triangle_moments(const double r[3], const double* P0, const double* P1, const double* P2, double& I0,
                               double Iv[3], double p[3], double n[3], double& area2) {
  double e1[3], e2[3], nn[3];
  sub(P1, P0, e1);
  sub(P2, P0, e2);
  cross(e1, e2, nn);
  area2 = sqrt(dot(nn, nn));
  for (int k = 0; k < 3; ++k) n[k] = nn[k] / area2;
  double rp[3];
  sub(r, P0, rp);
  const double d = dot(rp, n);
  for (int k = 0; k < 3; ++k) p[k] = r[k] - d * n[k];
  const double ad = fabs(d);
  const double tiny = 1e-13 * sqrt(area2);
  I0 = 0;
  Iv[0] = Iv[1] = Iv[2] = 0;
  const double* V[3] = {P0, P1, P2};
  for (int e = 0; e < 3; ++e) {
    const double* Pm = V[e];
    const double* Pp = V[(e + 1) % 3];
    double ev[3], l[3], u[3], a[3], b[3];
    sub(Pp, Pm, ev);
    const double le = sqrt(dot(ev, ev));
    for (int k = 0; k < 3; ++k) l[k] = ev[k] / le;
    cross(l, n, u);
    sub(Pm, p, a);
    sub(Pp, p, b);
    const double t = dot(a, u);
    const double lm = dot(a, l), lp = dot(b, l);
    const double R02 = t * t + d * d;
    double ra[3], rb[3];
    sub(Pm, r, ra);
    sub(Pp, r, rb);
    const double Rm = sqrt(dot(ra, ra)), Rp = sqrt(dot(rb, rb));
    double f = 0, at = 0;
    const bool ok = R02 > tiny * tiny;
    if (ok) {
      // R + l without cancellation: for l < 0 use R0^2 / (R - l)
      const double Ap = lp >= 0 ? Rp + lp : R02 / (Rp - lp);
      const double Am = lm >= 0 ? Rm + lm : R02 / (Rm - lm);
      f = log(Ap / Am);
      at = atan(t * lp / (R02 + ad * Rp)) - atan(t * lm / (R02 + ad * Rm));
      I0 += t * f - ad * at;
    }
    const double w = 0.5 * ((ok ? R02 * f : 0.0) + lp * Rp - lm * Rm);
    for (int k = 0; k < 3; ++k) Iv[k] += w * u[k];
  }
}

// int_tri phi_j / |r - r'| dS' for the three hat functions of triangle (a, b, c): a linear
// density integrates through its value at p and its in-plane gradient.
PMFEM_HD void tri_hat_potentials(const double r[3], const double a[3], const double b[3], const double c[3],
                                 double out[3]) {
  double I0, Iv[3], p[3], n[3], area2;
  triangle_moments(r, a, b, c, I0, Iv, p, n, area2);
  const double* V[3] = {a, b, c};
  for (int j = 0; j < 3; ++j) {
    const double* q1 = V[(j + 1) % 3];
    const double* q2 = V[(j + 2) % 3];
    double x1[3], x2[3], cr[3], e[3], g[3];
    sub(q1, p, x1);
    sub(q2, p, x2);
    cross(x1, x2, cr);
    const double lam = dot(cr, n) / area2;
    sub(q2, q1, e);
    cross(n, e, g);
    out[j] = lam * I0 + dot(g, Iv) / area2;
  }
}

// int_tet dV' / |r - r'|: div'((r'-r)/|r'-r|) = 2/|r'-r| turns the volume integral into
// 1/2 sum over faces of h_f int_f dS/R, h_f = (P_f - r).n_f with outward n_f.
PMFEM_HD double tet_potential(const double r[3], const double X[4][3]) {
  const int fc[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
  double cen[3] = {0, 0, 0};
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) cen[k] += 0.25 * X[i][k];
  double acc = 0;
  for (int f = 0; f < 4; ++f) {
    const double* A = X[fc[f][0]];
    const double* B = X[fc[f][1]];
    const double* C = X[fc[f][2]];
    double e1[3], e2[3], nn[3], ac[3];
    sub(B, A, e1);
    sub(C, A, e2);
    cross(e1, e2, nn);
    sub(A, cen, ac);
    if (dot(nn, ac) < 0) {
      const double* t = B;
      B = C;
      C = t;
    }
    double I0, Iv[3], p[3], n[3], area2;
    triangle_moments(r, A, B, C, I0, Iv, p, n, area2);
    double ar[3];
    sub(A, r, ar);
    acc += 0.5 * dot(ar, n) * I0;
  }
  return acc;
}

// ------------------------------------------------------------------ Lagrange stencil
// w_i(s) = prod_{j != i} (s - j)/(i - j), i = 0..p (order-p stencil, local coordinate s).
PMFEM_HD void lagrange(double sv, int p, double* w) {
  for (int i = 0; i <= p; ++i) {
    double v = 1.0;
    for (int j = 0; j <= p; ++j)
      if (j != i) v *= (sv - j) / (double)(i - j);
    w[i] = v;
  }
}

// ------------------------------------------------------------------ PGF of Eq. 15
// Parameters of one lattice (built on the host by PeriodicGreen); kvec points to nk rows of
// (kx, ky, kz, coefficient) in the memory of the side that evaluates (host or device).
struct PgfParams {
  int dim = 0;
  int ax[3] = {0, 1, 2};   // periodic axes first, then the open ones
  double L[3] = {0, 0, 0};
  int per[3] = {0, 0, 0};
  double eta = 0;
  int nimg[3] = {0, 0, 0};
  int nk = 0;
  const double* kvec = nullptr;
  double gl_u[kGaussLegendre] = {};
  double gl_w[kGaussLegendre] = {};
  int ngl = 0;
  double reg0 = 0;
};

// Ein(x) = int_0^x (1 - e^-t)/t dt: power series below 1, E1 + ln x + gamma above, with E1
// by the continued fraction of Abramowitz & Stegun 5.1.22 (modified Lentz).
PMFEM_HD double expint_e1_cf(double x) {
  const double tiny = 1e-300;
  double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 1000; ++i) {
    const double an = -(double)i * i;
    b += 2.0;
    d = 1.0 / (an * d + b);
    c = b + an / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}
PMFEM_HD double ein(double x) {
  if (x < 1.0) {
    double term = x, acc = x;
    for (int k = 2; k < 40; ++k) {
      term = -term * x / k;
      acc += term / k;
    }
    return acc;
  }
  return expint_e1_cf(x) + log(x) + kEulerGamma;
}

PMFEM_HD double pgf_real_space(const PgfParams& P, double x, double y, double z, bool skip_origin) {
  double acc = 0;
  const double cut = kCutReal / P.eta + 1e-300;
  for (int i = -P.nimg[0]; i <= P.nimg[0]; ++i)
    for (int j = -P.nimg[1]; j <= P.nimg[1]; ++j)
      for (int k = -P.nimg[2]; k <= P.nimg[2]; ++k) {
        if (skip_origin && !i && !j && !k) continue;
        const double dx = x + i * P.L[0], dy = y + j * P.L[1], dz = z + k * P.L[2];
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d > 1.5 * cut) continue;   // erfc below 1e-40
        acc += erfc(P.eta * d) / d;
      }
  return acc;
}

PMFEM_HD double pgf_g3(const PgfParams& P, double x, double y, double z) {
  double acc = pgf_real_space(P, x, y, z, false);
  for (int q = 0; q < P.nk; ++q) {
    const double* kv = P.kvec + 4 * q;
    acc += kv[3] * cos(kv[0] * x + kv[1] * y + kv[2] * z);
  }
  return acc - kPiD / (P.eta * P.eta * P.L[0] * P.L[1] * P.L[2]);
}

PMFEM_HD double pgf_g2(const PgfParams& P, double x, double y, double z) {
  const double r[3] = {x, y, z};
  const double ra = r[P.ax[0]], rb = r[P.ax[1]], zz = r[P.ax[2]];
  const double Ar = P.L[P.ax[0]] * P.L[P.ax[1]];
  double acc = pgf_real_space(P, x, y, z, false);
  for (int q = 0; q < P.nk; ++q) {
    const double* kv = P.kvec + 4 * q;
    const double kk = kv[2];
    double slab = 0;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      const double a = kk / (2 * P.eta) + sgn * P.eta * zz;
      const double t = erfc(a);
      if (t > 0) slab += exp(sgn * kk * zz + log(t));
    }
    acc += kv[3] * cos(kv[0] * ra + kv[1] * rb) * slab;
  }
  acc -= 2 * kPiD / Ar * (zz * erf(P.eta * zz) + exp(-P.eta * P.eta * zz * zz) / (P.eta * sqrt(kPiD)));
  return acc;
}

PMFEM_HD double pgf_g1(const PgfParams& P, double x, double y, double z) {
  const double r[3] = {x, y, z};
  const int a = P.ax[0];
  const double zz = r[a];
  const double rho2 = x * x + y * y + z * z - zz * zz;
  const double rho2c = rho2 > 0 ? rho2 : 0.0;
  const double Lz = P.L[a];
  double acc = pgf_real_space(P, x, y, z, false);
  acc += (2.0 * log(P.eta) - ein(P.eta * P.eta * rho2c)) / Lz;
  const double b = rho2c * P.eta * P.eta;
  for (int q = 0; q < P.nk; ++q) {
    const double* kv = P.kvec + 4 * q;
    const double aa = kv[0] * kv[0] / (4 * P.eta * P.eta);
    double f = 0;
    for (int i = 0; i < P.ngl; ++i) f += P.gl_w[i] * exp(-b * P.gl_u[i] - aa / P.gl_u[i]) / P.gl_u[i];
    acc += kv[3] * cos(kv[0] * zz) * f;
  }
  return acc;
}

// G^p(r) for r not on the lattice (min-imaged first); free space: 1/r.
PMFEM_HD double pgf_eval(const PgfParams& P, double x, double y, double z) {
  if (P.dim == 0) return 1.0 / sqrt(x * x + y * y + z * z);
  if (P.per[0]) x -= nearbyint(x / P.L[0]) * P.L[0];
  if (P.per[1]) y -= nearbyint(y / P.L[1]) * P.L[1];
  if (P.per[2]) z -= nearbyint(z / P.L[2]) * P.L[2];
  if (P.dim == 3) return pgf_g3(P, x, y, z);
  if (P.dim == 2) return pgf_g2(P, x, y, z);
  return pgf_g1(P, x, y, z);
}

}  // namespace sm
}  // namespace pmfem

namespace pmfem {
namespace sm {

// ------------------------------------------------------------------ near-element correction
// One row n of the Eq. 14c correction: for every near placement (element s translated by a
// lattice vector l) of the row, the exact integral of the element's source density minus its
// nodal point charges, as 3-vectors acting on the M of the element's vertices:
//   tetrahedron (uniform rho = -sum_j M_j.grad phi_j, point charges rho V/4):
//       coef = int_{s+l} dV'/|r_n - r'| - sum_i (V/4) G0'(r_n - r_i - l),   v_j = -grad phi_j coef
//   boundary triangle (linear sigma = M.n, point charges (A/12)(2 sigma_k + sum_{j!=k} sigma_j)):
//       coef_j = int_{s+l} phi_j dS'/|r_n - r'| - (A/12)(sum_i G_i + G_j),       v_j = n coef_j
// with G0'(0) = 0 for the vertex that is the observer itself.  Contributions are added, in the
// order of the row's placements, to out[3 * dest + d]; each placement lists the destination
// slot of every vertex (slots of one row are the row's own).
struct NearArgs {
  const double* xyz;      // N x 3 original node coordinates
  const int32_t* tets;    // T x 4
  const int32_t* bfaces;  // F x 3 boundary triangles (outward)
  const int32_t* lca;     // N: node -> unknown
  const double* pos_f;    // Np x 3 folded unknown positions
  double L[3];            // periods (0 on open axes)
  int64_t T;              // tetrahedra; element ids >= T are boundary triangles
  double self_tol;        // a vertex within this distance of its own unknown is the observer
  const int64_t* pptr;    // Np + 1: placements of each row
  const int64_t* elem;    // per placement
  const int32_t* img;     // 3 per placement: lattice vector in periods
  const int64_t* dest;    // 4 per placement: output slot of each vertex's 3-vector
};

PMFEM_HD void near_eval_row(const NearArgs& A, int64_t n, double* out) {
  const double* rn = A.pos_f + 3 * n;
  for (int64_t q = A.pptr[n]; q < A.pptr[n + 1]; ++q) {
    double obs[3];
    for (int d = 0; d < 3; ++d) obs[d] = rn[d] - A.img[3 * q + d] * A.L[d];
    const int64_t el = A.elem[q];
    const int64_t* dst = A.dest + 4 * q;
    if (el < A.T) {
      double X[4][3], g[4][3];
      int32_t vid[4];
      for (int i = 0; i < 4; ++i) {
        vid[i] = A.tets[4 * el + i];
        for (int d = 0; d < 3; ++d) X[i][d] = A.xyz[3 * (int64_t)vid[i] + d];
      }
      const double Ve = tet_grads(X, g);
      const double I = tet_potential(obs, X);
      double Ppt = 0;
      for (int i = 0; i < 4; ++i) {
        const double d0 = obs[0] - X[i][0], d1 = obs[1] - X[i][1], d2 = obs[2] - X[i][2];
        const double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const bool self = A.lca[vid[i]] == n && dist < A.self_tol;
        if (!self) Ppt += 0.25 * Ve / dist;
      }
      const double coef = I - Ppt;
      for (int j = 0; j < 4; ++j)
        for (int d = 0; d < 3; ++d) out[3 * dst[j] + d] += -g[j][d] * coef;
    } else {
      const int64_t f = el - A.T;
      int32_t vid[3];
      double X[3][3];
      for (int i = 0; i < 3; ++i) {
        vid[i] = A.bfaces[3 * f + i];
        for (int d = 0; d < 3; ++d) X[i][d] = A.xyz[3 * (int64_t)vid[i] + d];
      }
      double e1[3], e2[3], nn[3];
      sub(X[1], X[0], e1);
      sub(X[2], X[0], e2);
      cross(e1, e2, nn);
      const double a2 = sqrt(dot(nn, nn));
      const double nrm[3] = {nn[0] / a2, nn[1] / a2, nn[2] / a2};
      const double area = 0.5 * a2;
      double Ij[3];
      tri_hat_potentials(obs, X[0], X[1], X[2], Ij);
      double G[3], Gs = 0;
      for (int i = 0; i < 3; ++i) {
        const double d0 = obs[0] - X[i][0], d1 = obs[1] - X[i][1], d2 = obs[2] - X[i][2];
        const double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const bool self = A.lca[vid[i]] == n && dist < A.self_tol;
        G[i] = self ? 0.0 : 1.0 / dist;
        Gs += G[i];
      }
      for (int j = 0; j < 3; ++j) {
        const double coef = Ij[j] - area / 12.0 * (Gs + G[j]);
        for (int d = 0; d < 3; ++d) out[3 * dst[j] + d] += nrm[d] * coef;
      }
    }
  }
}

// ------------------------------------------------------------------ point precorrection
// Value of one box-near pair (observer n, source k, source image img in periods) of BAIM
// step 4: the exact point interaction G0(r_n - r_k - l) (0 for the self pair) minus what the
// grid carries, sum_a sum_b w_na w_kb G0'(r_a - r_b - l), computed as the separable
// correlation c of the two stencils per axis followed by a sum over the table T0 of G0' on
// integer grid offsets within R of zero (width W = 2R + 1).
PMFEM_HD double precorr_value(const double* rn, const double* rk, const int img[3], const double L[3],
                              const int Dbase[3], const double wn[3][6], const double* frack, int p, const int dimN[3],
                              const double* T0, int R, bool self) {
  const int P = p + 1, W = 2 * R + 1;
  double val = 0;
  if (!self) {
    const double d0 = rn[0] - rk[0] - img[0] * L[0];
    const double d1 = rn[1] - rk[1] - img[1] * L[1];
    const double d2 = rn[2] - rk[2] - img[2] * L[2];
    val = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  }
  double wk[3][6], c[3][11];
  int D[3];
  for (int a = 0; a < 3; ++a) {
    lagrange(frack[a], p, wk[a]);
    D[a] = Dbase[a] - img[a] * dimN[a];
    for (int i = 0; i < 2 * p + 1; ++i) c[a][i] = 0;
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) c[a][i - j + p] += wn[a][i] * wk[a][j];
  }
  double gsum = 0;
  for (int tz = 0; tz <= 2 * p; ++tz) {
    const int64_t oz2 = (int64_t)W * W * (D[2] + tz - p + R);
    double sy = 0;
    for (int ty = 0; ty <= 2 * p; ++ty) {
      const int64_t oy2 = oz2 + (int64_t)W * (D[1] + ty - p + R);
      double sx = 0;
      for (int tx = 0; tx <= 2 * p; ++tx) sx += c[0][tx] * T0[oy2 + (D[0] + tx - p + R)];
      sy += c[1][ty] * sx;
    }
    gsum += c[2][tz] * sy;
  }
  return val - gsum;
}

}  // namespace sm
}  // namespace pmfem

namespace pmfem {
namespace sm {

// ------------------------------------------------------------------ Bloch-phase PGF
// Eq. 15 with a phase per image, G_k(r) = sum_l e^{-j k0.l} / |r - l|, by Ewald splitting:
// real-space images with their phases, then the smooth part summed over the shifted reciprocal
// vectors g = G + k0 (kv rows: gx, gy, gz, coefficient): 3D coefficient (4 pi/V) e^{-g^2/4eta^2}/g^2;
// 2D (pi/A)/|g| times the slab function of the open coordinate; 1D 1/L times
// int_0^{eta^2} exp(-rho^2 s - g^2/4s) ds/s, summed with s = eta^2 e^{-t} by 16-point
// Gauss-Legendre on unit panels of t (the rule stays accurate for the small |g| near k0).
struct BlochParams {
  int dim = 0;
  int ax[3] = {0, 1, 2};
  double L[3] = {0, 0, 0};
  double k0[3] = {0, 0, 0};
  double eta = 0;
  int nimg[3] = {0, 0, 0};
  int nk = 0;
  const double* kv = nullptr;   // nk x 4
  double gl_x[16] = {}, gl_w[16] = {};
};

PMFEM_HD double bloch_spectral_1d(double rho, double k, double eta, const double* glx, const double* glw) {
  const double a = k * k / (4.0 * eta * eta), b = rho * rho * eta * eta;
  const double T = a < 45.0 ? fmax(1.0, log(45.0 / a) + 1.0) : 1.0;
  const int npan = (int)ceil(T);
  double out = 0;
  for (int p = 0; p < npan; ++p)
    for (int i = 0; i < 16; ++i) {
      const double t = p + 0.5 * (glx[i] + 1.0);
      out += 0.5 * glw[i] * exp(-b * exp(-t) - a * exp(t));
    }
  return out;
}

// Real-space part of G_k(r): the images within reach of erfc, each with its phase; skip_origin
// drops the l = 0 image (for the regular part at r = 0)
PMFEM_HD void bloch_real_part(const BlochParams& P, double x, double y, double z, bool skip_origin, double* re,
                              double* im) {
  double sr = 0, si = 0;
  const double cut = kCutReal / P.eta;
  for (int i = -P.nimg[0]; i <= P.nimg[0]; ++i)
    for (int j = -P.nimg[1]; j <= P.nimg[1]; ++j)
      for (int k = -P.nimg[2]; k <= P.nimg[2]; ++k) {
        if (skip_origin && !i && !j && !k) continue;
        const double lx = i * P.L[0], ly = j * P.L[1], lz = k * P.L[2];
        const double dx = x - lx, dy = y - ly, dz = z - lz;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d > 1.5 * cut) continue;
        const double t = erfc(P.eta * d) / d;
        const double ph = -(P.k0[0] * lx + P.k0[1] * ly + P.k0[2] * lz);
        sr += t * cos(ph);
        si += t * sin(ph);
      }
  *re = sr;
  *im = si;
}

// Amplitude of spectral term q at r, without its phase e^{-j g.r}: the coefficient times, in 2D,
// the slab function of the open coordinate and, in 1D, the radial integral at the distance from
// the lattice axis.  It depends on r only through that coordinate (2D) or distance (1D).
PMFEM_HD double bloch_term_amp(const BlochParams& P, int q, double x, double y, double z) {
  const double r[3] = {x, y, z};
  const double* g = P.kv + 4 * q;
  double amp = g[3];
  if (P.dim == 2) {
    const double kk = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const double zz = r[P.ax[2]];
    double slab = 0;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      const double e = erfc(kk / (2 * P.eta) + sgn * P.eta * zz);
      if (e > 0) slab += exp(sgn * kk * zz + log(e));
    }
    amp *= slab;
  } else if (P.dim == 1) {
    const int a = P.ax[0];
    const double rho2 = x * x + y * y + z * z - r[a] * r[a];
    amp *= bloch_spectral_1d(sqrt(rho2 > 0 ? rho2 : 0.0), fabs(g[a]), P.eta, P.gl_x, P.gl_w);
  }
  return amp;
}

// G_k(r) = real-space part + sum over the shifted reciprocal vectors of amplitude x e^{-j g.r}
PMFEM_HD void bloch_eval(const BlochParams& P, double x, double y, double z, bool skip_origin, double* re,
                         double* im) {
  double sr, si;
  bloch_real_part(P, x, y, z, skip_origin, &sr, &si);
  for (int q = 0; q < P.nk; ++q) {
    const double* g = P.kv + 4 * q;
    const double ph = -(g[0] * x + g[1] * y + g[2] * z);
    const double amp = bloch_term_amp(P, q, x, y, z);
    sr += amp * cos(ph);
    si += amp * sin(ph);
  }
  *re = sr;
  *im = si;
}

}  // namespace sm
}  // namespace pmfem
