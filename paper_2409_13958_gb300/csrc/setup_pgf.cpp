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
#include "setup_math.hpp"

namespace pmfem {

namespace {
using sm::kCutReal;
using sm::kCutSpec;
using sm::expint_e1_cf;

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
    gauss_legendre01(sm::kGaussLegendre, gl_u_, gl_w_);
  }
  fill_params();   // before the regular part, which evaluates the real-space sum
  // regular part at the origin
  double r = sm::pgf_real_space(P_, 0, 0, 0, true) - 2 * eta_ / std::sqrt(kPi);
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
  P_.reg0 = r;
}

void PeriodicGreen::fill_params() {
  P_ = sm::PgfParams();
  P_.dim = dim_;
  for (int a = 0; a < 3; ++a) {
    P_.ax[a] = ax_[a];
    P_.L[a] = L_[a];
    P_.per[a] = per_[a] ? 1 : 0;
    P_.nimg[a] = nimg_[a];
  }
  P_.eta = eta_;
  kflat_.clear();
  for (auto& kv : kvec_) kflat_.insert(kflat_.end(), kv.begin(), kv.end());
  P_.nk = (int)kvec_.size();
  P_.kvec = kflat_.data();
  P_.ngl = (int)gl_u_.size();
  for (int i = 0; i < P_.ngl; ++i) {
    P_.gl_u[i] = gl_u_[i];
    P_.gl_w[i] = gl_w_[i];
  }
}

double PeriodicGreen::operator()(double x, double y, double z) const { return sm::pgf_eval(P_, x, y, z); }

}  // namespace pmfem
