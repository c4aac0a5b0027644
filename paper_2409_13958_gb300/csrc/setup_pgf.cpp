// Periodic Green's function of Eq. 15 for k0 = 0 and G0 = 1/r, evaluated by Ewald-type
// splitting (the paper names exponentially convergent sums without details):
//   3D: sum_l erfc(eta|r+l|)/|r+l| + (4 pi/V) sum_{k!=0} e^{-k^2/4eta^2} cos(k.r)/k^2 - pi/(eta^2 V)
//   2D: sum_l erfc(eta|r+l|)/|r+l| + (pi/A) sum_{k!=0} cos(k.rho)/k [e^{kz} erfc(k/2eta+eta z)
//       + e^{-kz} erfc(k/2eta-eta z)] - (2 pi/A)[z erf(eta z) + e^{-eta^2 z^2}/(eta sqrt(pi))]
//   1D: sum_l erfc(eta r_l)/r_l + (1/L)[2 ln eta - Ein(eta^2 rho^2)]
//       + (2/L) sum_{j>=1} cos(k_j z) int_0^{eta^2} e^{-rho^2 s - k_j^2/4s} ds/s
// The k = 0 / constant parts are the ones that make the value independent of eta; every
// charge set summed with them is neutral, so constants never reach the field.
#include <cmath>

#include "internal.hpp"

namespace pmfem {

namespace {
constexpr double kCutReal = 6.3;   // erfc(6.3) ~ 1e-19
constexpr double kCutSpec = 43.0;  // exp(-43) ~ 2e-19
constexpr double kEuler = 0.57721566490153286061;

// E1(x) for x >= 1 by the continued fraction of Abramowitz & Stegun 5.1.22 (modified Lentz)
double expint_e1_cf(double x) {
  const double tiny = 1e-300;
  double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 1000; ++i) {
    double an = -(double)i * i;
    b += 2.0;
    d = 1.0 / (an * d + b);
    c = b + an / c;
    double del = c * d;
    h *= del;
    if (std::fabs(del - 1.0) < 1e-16) break;
  }
  return h * std::exp(-x);
}

// Ein(x) = int_0^x (1 - e^-t)/t dt: power series below 1, E1 + ln x + gamma above
double ein(double x) {
  if (x < 1.0) {
    double term = x, acc = x;
    for (int k = 2; k < 40; ++k) {
      term = -term * x / k;
      acc += term / k;
    }
    return acc;
  }
  return expint_e1_cf(x) + std::log(x) + kEuler;
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton iteration on P_n)
void gauss_legendre01(int n, std::vector<double>& u, std::vector<double>& w) {
  u.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1);
      double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    u[i] = 0.5 * (1.0 - x);
    w[i] = 1.0 / ((1 - x * x) * dp * dp);   // 2/((1-x^2)P'^2) on [-1,1], halved for [0,1]
  }
}
}  // namespace

PeriodicGreen::PeriodicGreen(const double L[3], double eta_scale) {
  int k = 0;
  double prod = 1;
  for (int a = 0; a < 3; ++a) {
    L_[a] = L[a];
    per_[a] = L[a] > 0;
    if (per_[a]) {
      ax_[k++] = a;
      prod *= L[a];
    }
  }
  dim_ = k;
  for (int a = 0; a < 3; ++a)
    if (!per_[a]) ax_[k++] = a;
  if (dim_ == 0) {
    reg0_ = 0;
    return;
  }
  eta_ = eta_scale * std::sqrt(kPi) / std::pow(prod, 1.0 / dim_);
  for (int a = 0; a < 3; ++a)
    nimg_[a] = per_[a] ? (int)std::ceil(kCutReal / (eta_ * L_[a]) + 0.5) + 1 : 0;
  const double kmax = 2.0 * eta_ * std::sqrt(kCutSpec);
  if (dim_ == 3) {
    const double V = L_[0] * L_[1] * L_[2];
    int n[3];
    for (int a = 0; a < 3; ++a) n[a] = (int)std::ceil(kmax * L_[a] / (2 * kPi));
    for (int i = -n[0]; i <= n[0]; ++i)
      for (int j = -n[1]; j <= n[1]; ++j)
        for (int l = -n[2]; l <= n[2]; ++l) {
          if (!i && !j && !l) continue;
          double kx = 2 * kPi * i / L_[0], ky = 2 * kPi * j / L_[1], kz = 2 * kPi * l / L_[2];
          double k2 = kx * kx + ky * ky + kz * kz;
          double c = 4 * kPi / V * std::exp(-k2 / (4 * eta_ * eta_)) / k2;
          if (c > 0) kvec_.push_back({kx, ky, kz, c});
        }
  } else if (dim_ == 2) {
    int pa = ax_[0], pb = ax_[1];
    const double Ar = L_[pa] * L_[pb];
    int na = (int)std::ceil(kmax * L_[pa] / (2 * kPi)), nb = (int)std::ceil(kmax * L_[pb] / (2 * kPi));
    for (int i = -na; i <= na; ++i)
      for (int j = -nb; j <= nb; ++j) {
        if (!i && !j) continue;
        double ka = 2 * kPi * i / L_[pa], kb = 2 * kPi * j / L_[pb];
        double kk = std::sqrt(ka * ka + kb * kb);
        kvec_.push_back({ka, kb, kk, kPi / Ar / kk});
      }
  } else {
    const double Lz = L_[ax_[0]];
    for (int j = 1;; ++j) {
      double kz = 2 * kPi * j / Lz;
      if (kz * kz / (4 * eta_ * eta_) > kCutSpec) break;
      kvec_.push_back({kz, 0, 0, 2.0 / Lz});
    }
    gauss_legendre01(48, gl_u_, gl_w_);
  }
  // regular part at the origin
  double r = real_space(0, 0, 0, true) - 2 * eta_ / std::sqrt(kPi);
  if (dim_ == 3) {
    const double V = L_[0] * L_[1] * L_[2];
    for (auto& kv : kvec_) r += kv[3];
    r -= kPi / (eta_ * eta_ * V);
  } else if (dim_ == 2) {
    const double Ar = L_[ax_[0]] * L_[ax_[1]];
    for (auto& kv : kvec_) r += kv[3] * 2.0 * std::erfc(kv[2] / (2 * eta_));
    r -= 2 * kPi / (Ar * eta_ * std::sqrt(kPi));
  } else {
    const double Lz = L_[ax_[0]];
    r += 2.0 * std::log(eta_) / Lz;
    for (auto& kv : kvec_) r += kv[3] * expint_e1_cf(kv[0] * kv[0] / (4 * eta_ * eta_));
  }
  reg0_ = r;
}

void PeriodicGreen::min_image(double& x, double& y, double& z) const {
  double* v[3] = {&x, &y, &z};
  for (int a = 0; a < 3; ++a)
    if (per_[a]) *v[a] -= std::nearbyint(*v[a] / L_[a]) * L_[a];
}

double PeriodicGreen::real_space(double x, double y, double z, bool skip_origin) const {
  double acc = 0;
  const double cut = kCutReal / eta_ + 1e-300;
  for (int i = -nimg_[0]; i <= nimg_[0]; ++i)
    for (int j = -nimg_[1]; j <= nimg_[1]; ++j)
      for (int k = -nimg_[2]; k <= nimg_[2]; ++k) {
        if (skip_origin && !i && !j && !k) continue;
        double dx = x + i * L_[0], dy = y + j * L_[1], dz = z + k * L_[2];
        double d = std::sqrt(dx * dx + dy * dy + dz * dz);
        if (d > 1.5 * cut) continue;   // erfc below 1e-40
        acc += std::erfc(eta_ * d) / d;
      }
  return acc;
}

double PeriodicGreen::g3(double x, double y, double z) const {
  double acc = real_space(x, y, z, false);
  for (auto& kv : kvec_) acc += kv[3] * std::cos(kv[0] * x + kv[1] * y + kv[2] * z);
  return acc - kPi / (eta_ * eta_ * L_[0] * L_[1] * L_[2]);
}

double PeriodicGreen::g2(double x, double y, double z) const {
  double r[3] = {x, y, z};
  const double ra = r[ax_[0]], rb = r[ax_[1]], zz = r[ax_[2]];
  const double Ar = L_[ax_[0]] * L_[ax_[1]];
  double acc = real_space(x, y, z, false);
  for (auto& kv : kvec_) {
    double kk = kv[2];
    double slab = 0;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      double a = kk / (2 * eta_) + sgn * eta_ * zz;
      double t = std::erfc(a);
      if (t > 0) slab += std::exp(sgn * kk * zz + std::log(t));
    }
    acc += kv[3] * std::cos(kv[0] * ra + kv[1] * rb) * slab;
  }
  acc -= 2 * kPi / Ar * (zz * std::erf(eta_ * zz) + std::exp(-eta_ * eta_ * zz * zz) / (eta_ * std::sqrt(kPi)));
  return acc;
}

double PeriodicGreen::g1(double x, double y, double z) const {
  double r[3] = {x, y, z};
  const int a = ax_[0];
  const double zz = r[a];
  const double rho2 = x * x + y * y + z * z - zz * zz;
  const double rho2c = rho2 > 0 ? rho2 : 0.0;
  const double Lz = L_[a];
  double acc = real_space(x, y, z, false);
  acc += (2.0 * std::log(eta_) - ein(eta_ * eta_ * rho2c)) / Lz;
  const double b = rho2c * eta_ * eta_;
  for (auto& kv : kvec_) {
    const double aa = kv[0] * kv[0] / (4 * eta_ * eta_);
    double f = 0;
    for (size_t i = 0; i < gl_u_.size(); ++i) f += gl_w_[i] * std::exp(-b * gl_u_[i] - aa / gl_u_[i]) / gl_u_[i];
    acc += kv[3] * std::cos(kv[0] * zz) * f;
  }
  return acc;
}

double PeriodicGreen::operator()(double x, double y, double z) const {
  if (dim_ == 0) return 1.0 / std::sqrt(x * x + y * y + z * z);
  min_image(x, y, z);
  if (dim_ == 3) return g3(x, y, z);
  if (dim_ == 2) return g2(x, y, z);
  return g1(x, y, z);
}

}  // namespace pmfem
