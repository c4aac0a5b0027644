// Bloch-phase PGF on the GPU (bloch.cu): parameters, the FP64 spectrum of the twisted grid
// kernel, and the grid convolution of quasi-periodic sources.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.hpp"
#include "setup_math.hpp"

namespace pmfem {

// Ewald parameters of G_k on the handle's lattice (host); EINVAL for k0 off the periodic axes,
// no periodic axis, or k0 on the reciprocal lattice
int bloch_params(const Setup& s, const double k0[3], sm::BlochParams& P, std::vector<double>& kv, Error& err);
// spectrum of the twisted kernel on the FFT grid (F0 F1 F2 doubles on the device, x fastest,
// unscaled) and the largest |imaginary part| of the transform (zero up to rounding)
int bloch_spectrum_device(const Setup& s, const double k0[3], double* spec_dev, double* max_imag, Error& err);
// U~ = IFFT(spec FFT(pad(Q~))) cropped to the node grid; Q, U complex interleaved N0 N1 N2 of T;
// buf complex scratch of F0 F1 F2 elements; tw[a] = exp(-2 pi i j / F_a) in T (the handle's tables)
template <typename T>
void bloch_convolve_device(const Setup& s, const T* spec, const void* Q, void* U, void* buf,
                           const void* const tw[3], cudaStream_t st);

// fft.cu: BAIM step 2 for the twisted kernel with the line transforms of the k0 = 0 path, complex
// to complex over the full FFT grid (five passes: x forward on the populated rows, y forward on
// the populated planes, z forward + multiply by the full real spectrum + z inverse, y inverse, x
// inverse scaled by 1 / (F0 F1 F2)); Q, U complex N0 N1 N2 (x fastest), cb complex scratch of
// F0 F1 F2 elements (never cleared: zero inputs are not read), spec F0 F1 F2 (x fastest, unscaled)
template <typename T, typename C2>
void launch_bloch_fft_conv(const C2* Q, C2* U, C2* cb, const T* spec, const int dims[3], const int fft[3],
                           const C2* const tw[3], cudaStream_t st);
// fft.cu: in-place forward transform of a complex F0 F1 F2 grid (x fastest) in FP64
void launch_fft3_forward_f64(double2* buf, const int fft[3], const double2* const tw[3], cudaStream_t st);

}  // namespace pmfem
