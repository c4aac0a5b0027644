// Exact potential integrals used by the near-field correction of Sec. 3.2 (Eq. 14c): host
// entry points of the closed forms in setup_math.hpp (shared with the GPU set-up).
#include <cmath>

#include "internal.hpp"
#include "setup_math.hpp"

namespace pmfem {

void tri_hat_potentials(const double r[3], const double a[3], const double b[3], const double c[3], double out[3]) {
  sm::tri_hat_potentials(r, a, b, c, out);
}

double tet_potential(const double r[3], const double X[4][3]) { return sm::tet_potential(r, X); }

}  // namespace pmfem
