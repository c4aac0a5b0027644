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
// buf_a/b/c complex scratch of F0 F1 F2 elements each
template <typename T>
void bloch_convolve_device(const Setup& s, const T* spec, const void* Q, void* U, void* buf_a, void* buf_b,
                           void* buf_c, cudaStream_t st);

}  // namespace pmfem
