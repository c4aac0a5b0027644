// Exact potential integrals used by the near-field correction of Sec. 3.2 (Eq. 14c).
// Triangle (unit normal n, observer r, its projection p on the plane, height d): with
// every edge taken counter-clockwise about n from P- to P+, direction l, in-plane
// outward normal u = l x n, t = (P- - p).u, l+- = (P+- - p).l, R0^2 = t^2 + d^2,
// R+- = |P+- - r| and f = ln((R+ + l+)/(R- + l-)), integrating 1/R in polar form about p
// edge by edge gives
//   int dS/R        = sum [t f - |d| (atan(t l+/(R0^2+|d|R+)) - atan(t l-/(R0^2+|d|R-)))]
//   int (r'-p)/R dS = 1/2 sum u [R0^2 f + l+ R+ - l- R-]
// and a linear density integrates through its value at p and its in-plane gradient.
// Tetrahedron, uniform density: div'((r'-r)/|r'-r|) = 2/|r'-r| turns the volume integral
// into 1/2 sum over faces of h_f int_f dS/R, h_f = (P_f - r).n_f with outward n_f.
#include <cmath>

#include "internal.hpp"

namespace pmfem {
namespace {
inline void sub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
inline double dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// I0 = int dS/R and Iv = int (r' - p)/R dS; also returns p and the unit normal
void triangle_moments(const double r[3], const double* P0, const double* P1, const double* P2,
                      double& I0, double Iv[3], double p[3], double n[3], double& area2) {
  double e1[3], e2[3], nn[3];
  sub(P1, P0, e1);
  sub(P2, P0, e2);
  cross(e1, e2, nn);
  area2 = std::sqrt(dot(nn, nn));
  for (int k = 0; k < 3; ++k) n[k] = nn[k] / area2;
  double rp[3];
  sub(r, P0, rp);
  const double d = dot(rp, n);
  for (int k = 0; k < 3; ++k) p[k] = r[k] - d * n[k];
  const double ad = std::fabs(d);
  const double tiny = 1e-13 * std::sqrt(area2);
  I0 = 0;
  Iv[0] = Iv[1] = Iv[2] = 0;
  const double* V[3] = {P0, P1, P2};
  for (int e = 0; e < 3; ++e) {
    const double* Pm = V[e];
    const double* Pp = V[(e + 1) % 3];
    double ev[3], l[3], u[3], a[3], b[3];
    sub(Pp, Pm, ev);
    double le = std::sqrt(dot(ev, ev));
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
    const double Rm = std::sqrt(dot(ra, ra)), Rp = std::sqrt(dot(rb, rb));
    double f = 0, at = 0;
    const bool ok = R02 > tiny * tiny;
    if (ok) {
      // R + l without cancellation: for l < 0 use R0^2 / (R - l)
      double Ap = lp >= 0 ? Rp + lp : R02 / (Rp - lp);
      double Am = lm >= 0 ? Rm + lm : R02 / (Rm - lm);
      f = std::log(Ap / Am);
      at = std::atan(t * lp / (R02 + ad * Rp)) - std::atan(t * lm / (R02 + ad * Rm));
      I0 += t * f - ad * at;
    }
    const double w = 0.5 * ((ok ? R02 * f : 0.0) + lp * Rp - lm * Rm);
    for (int k = 0; k < 3; ++k) Iv[k] += w * u[k];
  }
}
}  // namespace

void tri_hat_potentials(const double r[3], const double a[3], const double b[3], const double c[3], double out[3]) {
  double I0, Iv[3], p[3], n[3], area2;
  triangle_moments(r, a, b, c, I0, Iv, p, n, area2);
  const double* V[3] = {a, b, c};
  for (int j = 0; j < 3; ++j) {
    const double* q1 = V[(j + 1) % 3];
    const double* q2 = V[(j + 2) % 3];
    // barycentric coordinate of vertex j at p and its (in-plane) gradient
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

double tet_potential(const double r[3], const double X[4][3]) {
  static const int fc[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
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
    if (dot(nn, ac) < 0) std::swap(B, C);
    double I0, Iv[3], p[3], n[3], area2;
    triangle_moments(r, A, B, C, I0, Iv, p, n, area2);
    double ar[3];
    sub(A, r, ar);
    acc += 0.5 * dot(ar, n) * I0;
  }
  return acc;
}

}  // namespace pmfem
