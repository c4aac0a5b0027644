// Bloch-phase PGF (Eq. 15 with k0 != 0) on the GPU: the twisted grid kernel in FP64 by the
// Ewald-type sums, its spectrum, and the grid convolution of BAIM step 2 for sources that repeat
// with the phase e^{-j k0.l} (phase-shifted excitation, Sec. 4.3).
//
// With q~ = q e^{j k0.r} and K~(d) = G_k(d) e^{j k0.d}, which is periodic and Hermitian, the
// quasi-periodic potential is e^{-j k0.r} times the circular convolution of q~ with K~ on the grid
// of Eq. 16 (open axes zero-padded to 2N as for k0 = 0); the spectrum of a Hermitian kernel is
// real but, unlike the k0 = 0 spectrum, not even, so it is kept on the full FFT grid.  Both
// transforms (the FP64 one of the kernel table and the convolution's, in the precision's type)
// run the radix-2 line transforms of the k0 = 0 path in fft.cu, complex to complex.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/pmfem.h"
#include "bloch.hpp"
#include "setup_math.hpp"

namespace pmfem {
namespace {

constexpr int kB = 256;
unsigned nblk(int64_t n) { return (unsigned)((n + kB - 1) / kB); }

struct GridDesc {
  int dims[3], fft[3], per[3];
  double delta[3];
};

// signed offset of FFT index j along an axis; false where the open-axis layout holds zero
__device__ __forceinline__ bool offset_of(const GridDesc& g, int a, int j, int* d) {
  const int N = g.dims[a];
  if (g.per[a]) {
    *d = j <= N / 2 ? j : j - N;
    return true;
  }
  if (j == N) return false;
  *d = j < N ? j : j - 2 * N;
  return true;
}

// Spectral amplitudes that do not depend on the position along the periodic axes, tabulated once
// per spectrum: in 1D per (term q, transverse offset t = jb + F_b jc over the two open axes
// b = ax[1], c = ax[2]); in 2D per (q, open-axis index t = jc, c = ax[2]).  amp[q nt + t]; zero
// where the open-axis layout holds no offset.
__global__ void k_bloch_amp(sm::BlochParams P, GridDesc g, int nt, double* __restrict__ amp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)P.nk * nt) return;
  const int q = (int)(i / nt), t = (int)(i % nt);
  double r[3] = {0.0, 0.0, 0.0};
  if (P.dim == 1) {
    const int b = P.ax[1], c = P.ax[2];
    int db, dc;
    if (!offset_of(g, b, t % g.fft[b], &db) || !offset_of(g, c, t / g.fft[b], &dc)) {
      amp[i] = 0.0;
      return;
    }
    r[b] = db * g.delta[b];
    r[c] = dc * g.delta[c];
  } else {
    const int c = P.ax[2];
    int dc;
    if (!offset_of(g, c, t, &dc)) {
      amp[i] = 0.0;
      return;
    }
    r[c] = dc * g.delta[c];
  }
  amp[i] = sm::bloch_term_amp(P, q, r[0], r[1], r[2]);
}

// The twisted kernel K~(d) = G_k(d) e^{j k0.d} at every FFT-grid offset.  K~(-d) is the conjugate
// of K~(d), and the offset of index j along an axis is minus that of F - j (mod F), so the thread
// of the smaller of two mirrored linear indices computes both; self-mirrored indices compute
// themselves.  amp: the tabulated amplitudes (1D, 2D) or null (3D: the coefficients themselves).
__global__ void k_bloch_table(sm::BlochParams P, GridDesc g, double r0re, double r0im, const double* __restrict__ amp,
                              int nt, double2* __restrict__ out) {
  const int64_t n = (int64_t)g.fft[0] * g.fft[1] * g.fft[2];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j[3] = {(int)(i % g.fft[0]), (int)((i / g.fft[0]) % g.fft[1]), (int)(i / ((int64_t)g.fft[0] * g.fft[1]))};
  int mj[3];
  for (int a = 0; a < 3; ++a) mj[a] = j[a] ? g.fft[a] - j[a] : 0;
  const int64_t im = mj[0] + (int64_t)g.fft[0] * (mj[1] + (int64_t)g.fft[1] * mj[2]);
  if (im < i) return;
  int dx, dy, dz;
  double2 v = make_double2(0.0, 0.0);
  if (!offset_of(g, 0, j[0], &dx) || !offset_of(g, 1, j[1], &dy) || !offset_of(g, 2, j[2], &dz)) {
    // no offset here, nor at the mirror
  } else if (!dx && !dy && !dz) {
    v = make_double2(r0re, r0im);
  } else {
    const double x = dx * g.delta[0], y = dy * g.delta[1], z = dz * g.delta[2];
    double re, imv;
    sm::bloch_real_part(P, x, y, z, false, &re, &imv);
    int t = 0;
    if (P.dim == 1) t = j[P.ax[1]] + g.fft[P.ax[1]] * j[P.ax[2]];
    else if (P.dim == 2) t = j[P.ax[2]];
    for (int q = 0; q < P.nk; ++q) {
      const double* gv = P.kv + 4 * q;
      const double ph = -(gv[0] * x + gv[1] * y + gv[2] * z);
      const double a = amp ? amp[(int64_t)q * nt + t] : gv[3];
      re += a * cos(ph);
      imv += a * sin(ph);
    }
    const double ph = P.k0[0] * x + P.k0[1] * y + P.k0[2] * z;   // the twist e^{j k0.d}
    const double c = cos(ph), s = sin(ph);
    v = make_double2(re * c - imv * s, re * s + imv * c);
  }
  out[i] = v;
  if (im != i) out[im] = make_double2(v.x, -v.y);
}

__global__ void k_real_part(const double2* __restrict__ in, double* __restrict__ re, double* __restrict__ im_abs,
                            int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  re[i] = in[i].x;
  im_abs[i] = fabs(in[i].y);
}

GridDesc desc(const Setup& s) {
  GridDesc g;
  for (int a = 0; a < 3; ++a) {
    g.dims[a] = s.dims[a];
    g.fft[a] = s.fft[a];
    g.per[a] = s.periodic[a] ? 1 : 0;
    g.delta[a] = s.delta[a];
  }
  return g;
}

}  // namespace

int bloch_params(const Setup& s, const double k0[3], sm::BlochParams& P, std::vector<double>& kv, Error& err) {
  int dim = 0;
  double prod = 1;
  P = sm::BlochParams();
  for (int a = 0; a < 3; ++a) {
    P.L[a] = s.periodic[a] ? s.L[a] : 0.0;
    if (s.periodic[a]) {
      P.ax[dim++] = a;
      prod *= s.L[a];
    } else if (k0[a] != 0) {
      err = {EINVAL_, "k0 must lie along the periodic axes"};
      return EINVAL_;
    }
    P.k0[a] = k0[a];
  }
  if (dim == 0) {
    err = {EINVAL_, "the Bloch-phase Green's function needs a periodic axis"};
    return EINVAL_;
  }
  int k = dim;
  for (int a = 0; a < 3; ++a)
    if (!s.periodic[a]) P.ax[k++] = a;
  P.dim = dim;
  P.eta = std::sqrt(kPi) / std::pow(prod, 1.0 / dim);
  // off the reciprocal lattice: no shifted wavevector may vanish
  for (int a = 0; a < 3; ++a)
    if (s.periodic[a]) {
      const double f = k0[a] * s.L[a] / (2 * kPi);
      if (std::fabs(f - std::nearbyint(f)) < 1e-9 && dim > 0) {
        bool all = true;
        for (int b = 0; b < 3; ++b)
          if (s.periodic[b]) {
            const double fb = k0[b] * s.L[b] / (2 * kPi);
            all = all && std::fabs(fb - std::nearbyint(fb)) < 1e-9;
          }
        if (all) {
          err = {EINVAL_, "k0 on the reciprocal lattice: use the k0 = 0 path"};
          return EINVAL_;
        }
      }
    }
  for (int a = 0; a < 3; ++a) {
    if (!s.periodic[a]) continue;
    const double ext = 0.5 * s.L[a];   // table offsets reach half a period along a periodic axis
    P.nimg[a] = (int)std::ceil((sm::kCutReal / P.eta + ext) / s.L[a]) + 1;
  }
  const double kmax = 2.0 * P.eta * std::sqrt(sm::kCutSpec);
  int nr[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a)
    if (s.periodic[a]) nr[a] = (int)std::ceil((kmax + std::fabs(k0[a])) * s.L[a] / (2 * kPi)) + 1;
  kv.clear();
  double V = 1;
  for (int a = 0; a < dim; ++a) V *= s.L[P.ax[a]];
  for (int i = -nr[0]; i <= nr[0]; ++i)
    for (int j = -nr[1]; j <= nr[1]; ++j)
      for (int l = -nr[2]; l <= nr[2]; ++l) {
        const int idx[3] = {i, j, l};
        double g[3];
        for (int a = 0; a < 3; ++a) g[a] = (s.periodic[a] ? 2 * kPi * idx[a] / s.L[a] : 0.0) + k0[a];
        const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        if (g2 / (4 * P.eta * P.eta) > sm::kCutSpec) continue;
        double c;
        if (dim == 3) c = 4 * kPi / V * std::exp(-g2 / (4 * P.eta * P.eta)) / g2;
        else if (dim == 2) c = kPi / V / std::sqrt(g2);
        else c = 1.0 / V;
        kv.insert(kv.end(), {g[0], g[1], g[2], c});
      }
  P.nk = (int)(kv.size() / 4);
  // 16-point Gauss-Legendre on [-1, 1] (Newton on P_16)
  for (int i = 0; i < 16; ++i) {
    double x = std::cos(kPi * (i + 0.75) / 16.5), dp = 1;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = x;
      for (int kk = 2; kk <= 16; ++kk) {
        const double p2 = ((2 * kk - 1) * x * p1 - (kk - 1) * p0) / kk;
        p0 = p1;
        p1 = p2;
      }
      dp = 16 * (x * p1 - p0) / (x * x - 1);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    P.gl_x[i] = x;
    P.gl_w[i] = 2.0 / ((1 - x * x) * dp * dp);
  }
  return OK;
}

int bloch_spectrum_device(const Setup& s, const double k0[3], double* spec_dev, double* max_imag, Error& err) {
  sm::BlochParams P;
  std::vector<double> kv;
  int rc = bloch_params(s, k0, P, kv, err);
  if (rc) return rc;
  const GridDesc g = desc(s);
  const int64_t n = (int64_t)g.fft[0] * g.fft[1] * g.fft[2];
  double* dkv = nullptr;
  double2* a = nullptr;
  double* im = nullptr;
  double* amp = nullptr;
  double2* tw[3] = {nullptr, nullptr, nullptr};
  auto cleanup = [&]() {
    cudaFree(dkv);
    cudaFree(a);
    cudaFree(im);
    cudaFree(amp);
    for (double2* t : tw) cudaFree(t);
  };
  // amplitude table: 1D per (term, transverse offset), 2D per (term, open index), 3D none
  const int nt = P.dim == 1 ? g.fft[P.ax[1]] * g.fft[P.ax[2]] : P.dim == 2 ? g.fft[P.ax[2]] : 0;
  const int64_t namp = (int64_t)P.nk * nt;
  cudaError_t e = cudaMalloc(&dkv, std::max<size_t>(kv.size(), 4) * sizeof(double));
  if (e == cudaSuccess && namp > 0) e = cudaMalloc(&amp, namp * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&a, n * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&im, n * sizeof(double));
  if (e == cudaSuccess && !kv.empty()) e = cudaMemcpy(dkv, kv.data(), kv.size() * sizeof(double), cudaMemcpyHostToDevice);
  for (int ax = 0; ax < 3 && e == cudaSuccess; ++ax) {   // exp(-2 pi i j / F) in FP64
    const int F = g.fft[ax];
    std::vector<double2> t(F);
    for (int j = 0; j < F; ++j) t[j] = make_double2(std::cos(2.0 * kPi * j / F), -std::sin(2.0 * kPi * j / F));
    e = cudaMalloc(&tw[ax], F * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(tw[ax], t.data(), F * sizeof(double2), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cleanup();
    err = {ECUDA_, std::string("Bloch spectrum: ") + cudaGetErrorString(e)};
    return ECUDA_;
  }
  P.kv = dkv;
  // regular part at the origin: the image sum without l = 0, minus the Gaussian self term
  double r0re = 0, r0im = 0;
  {
    std::vector<double> hk = kv;
    sm::BlochParams Ph = P;
    Ph.kv = hk.data();
    sm::bloch_eval(Ph, 0, 0, 0, true, &r0re, &r0im);
    r0re -= 2 * P.eta / std::sqrt(kPi);
  }
  if (namp > 0) k_bloch_amp<<<nblk(namp), kB>>>(P, g, nt, amp);
  k_bloch_table<<<nblk(n), kB>>>(P, g, r0re, r0im, amp, nt, a);
  const double2* twc[3] = {tw[0], tw[1], tw[2]};
  launch_fft3_forward_f64(a, g.fft, twc, 0);
  k_real_part<<<nblk(n), kB>>>(a, spec_dev, im, n);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  double mi = 0;
  if (e == cudaSuccess && max_imag) {
    std::vector<double> h(n);
    e = cudaMemcpy(h.data(), im, n * sizeof(double), cudaMemcpyDeviceToHost);
    for (double v : h) mi = std::max(mi, v);
    *max_imag = mi;
  }
  cleanup();
  if (e != cudaSuccess) {
    err = {ECUDA_, std::string("Bloch spectrum kernels: ") + cudaGetErrorString(e)};
    return ECUDA_;
  }
  return OK;
}

template <typename T>
void bloch_convolve_device(const Setup& s, const T* spec, const void* Q, void* U, void* buf,
                           const void* const tw[3], cudaStream_t st) {
  using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  const GridDesc g = desc(s);
  const C* twc[3] = {(const C*)tw[0], (const C*)tw[1], (const C*)tw[2]};
  launch_bloch_fft_conv<T, C>((const C*)Q, (C*)U, (C*)buf, spec, g.dims, g.fft, twc, st);
}

template void bloch_convolve_device<double>(const Setup&, const double*, const void*, void*, void*,
                                            const void* const*, cudaStream_t);
template void bloch_convolve_device<float>(const Setup&, const float*, const void*, void*, void*,
                                           const void* const*, cudaStream_t);

}  // namespace pmfem
