// BAIM step 2 on sm_103a: U = IFFT( Ghat . FFT(Q) ) over the grid of Eq. 16.
// Periodic axes are transformed circularly at their own length; open axes are zero-padded
// to twice their length (linear convolution).  Five passes over a complex half-spectrum
// buffer laid out [z][y][kx] (kx = 0..F0/2):
//   1. x: real-to-complex on the N1 x N2 populated rows (inputs beyond N0 are zero)
//   2. y: forward on the populated z planes, inputs beyond N1 are zero
//   3. z: forward (inputs beyond N2 zero), multiply by the real PGF spectrum, inverse,
//         keep z < N2
//   4. y: inverse on the populated z planes, keep y < N1
//   5. x: complex-to-real on the kept rows, keep x < N0
// Each line transform is an in-shared-memory Stockham radix-2 (autosort) FFT; a block
// takes BL lines that are adjacent in memory so that loads and stores coalesce.
#include "device.hpp"

namespace pmfem {
namespace {

constexpr int kThreads = 256;
constexpr int kSmemBudget = 96 * 1024;

template <typename C2> __device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.x + b.x, a.y + b.y}; }
template <typename C2> __device__ __forceinline__ C2 csub(C2 a, C2 b) { return {a.x - b.x, a.y - b.y}; }
template <typename C2> __device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// BL lines of length F in x (line-major); returns the buffer holding the result.
template <typename C2>
__device__ C2* fft_lines(C2* x, C2* y, int F, int BL, const C2* __restrict__ tw, bool inverse) {
  const int H = F >> 1;
  for (int s = 1, m = F; m > 1; s <<= 1, m >>= 1) {
    const int half = m >> 1;
    for (int b = threadIdx.x; b < BL * H; b += blockDim.x) {
      const int l = b / H, i = b - l * H;
      const int p = i / s, q = i - p * s;
      C2* xl = x + l * F;
      C2* yl = y + l * F;
      const C2 a = xl[q + s * p], c = xl[q + s * (p + half)];
      C2 w = tw[p * s];
      if (inverse) w.y = -w.y;
      yl[q + s * 2 * p] = cadd(a, c);
      yl[q + s * (2 * p + 1)] = cmul(csub(a, c), w);
    }
    __syncthreads();
    C2* t = x;
    x = y;
    y = t;
  }
  return x;
}

template <typename T, typename C2>
__global__ void __launch_bounds__(kThreads) k_fft_x_fwd(const T* __restrict__ Q, C2* __restrict__ cb, int N0, int N1,
                                                       int N2, int F0, int F1, int BL, const C2* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  C2* y = x + BL * F0;
  const int64_t nlines = (int64_t)N1 * N2;
  const int64_t L0 = (int64_t)blockIdx.x * BL;
  for (int idx = threadIdx.x; idx < BL * F0; idx += blockDim.x) {
    const int l = idx / F0, j = idx - l * F0;
    const int64_t L = L0 + l;
    T v = 0;
    if (L < nlines && j < N0) v = Q[j + (int64_t)N0 * L];
    x[idx] = {v, T(0)};
  }
  __syncthreads();
  C2* r = fft_lines(x, y, F0, BL, tw, false);
  const int Hx = F0 / 2 + 1;
  for (int idx = threadIdx.x; idx < BL * Hx; idx += blockDim.x) {
    const int l = idx / Hx, k = idx - l * Hx;
    const int64_t L = L0 + l;
    if (L < nlines) {
      const int64_t yy = L % N1, zz = L / N1;
      cb[k + (int64_t)Hx * (yy + (int64_t)F1 * zz)] = r[l * F0 + k];
    }
  }
}

template <typename C2>
__global__ void __launch_bounds__(kThreads) k_fft_y(C2* __restrict__ cb, int Hx, int F1, int nz, int n_in, int n_out,
                                                   int BL, bool inverse, const C2* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  C2* y = x + BL * F1;
  const int kxb = (Hx + BL - 1) / BL;
  const int z = blockIdx.x / kxb;
  const int kx0 = (blockIdx.x - z * kxb) * BL;
  C2* plane = cb + (int64_t)Hx * F1 * z;
  for (int idx = threadIdx.x; idx < BL * F1; idx += blockDim.x) {
    const int j = idx / BL, l = idx - j * BL;
    C2 v = {0, 0};
    if (kx0 + l < Hx && j < n_in) v = plane[kx0 + l + (int64_t)Hx * j];
    x[l * F1 + j] = v;
  }
  __syncthreads();
  C2* r = fft_lines(x, y, F1, BL, tw, inverse);
  for (int idx = threadIdx.x; idx < BL * n_out; idx += blockDim.x) {
    const int j = idx / BL, l = idx - j * BL;
    if (kx0 + l < Hx) plane[kx0 + l + (int64_t)Hx * j] = r[l * F1 + j];
  }
}

template <typename T, typename C2>
__global__ void __launch_bounds__(kThreads) k_fft_z_conv(C2* __restrict__ cb, int Hx, int F1, int F2, int N2, int BL,
                                                        const T* __restrict__ ghat, const C2* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  C2* y = x + BL * F2;
  const int kxb = (Hx + BL - 1) / BL;
  const int ky = blockIdx.x / kxb;
  const int kx0 = (blockIdx.x - ky * kxb) * BL;
  const int64_t zs = (int64_t)Hx * F1;
  C2* col0 = cb + kx0 + (int64_t)Hx * ky;
  for (int idx = threadIdx.x; idx < BL * F2; idx += blockDim.x) {
    const int j = idx / BL, l = idx - j * BL;
    C2 v = {0, 0};
    if (kx0 + l < Hx && j < N2) v = col0[l + zs * j];
    x[l * F2 + j] = v;
  }
  __syncthreads();
  C2* r = fft_lines(x, y, F2, BL, tw, false);
  C2* o = (r == x) ? y : x;
  const int H1 = F1 / 2 + 1;
  const int iy = ky <= F1 - ky ? ky : F1 - ky;
  for (int idx = threadIdx.x; idx < BL * F2; idx += blockDim.x) {
    const int l = idx / F2, j = idx - l * F2;
    const int kx = kx0 + l < Hx ? kx0 + l : Hx - 1;
    const int iz = j <= F2 - j ? j : F2 - j;
    const T g = ghat[kx + (int64_t)Hx * (iy + (int64_t)H1 * iz)];
    r[idx].x *= g;
    r[idx].y *= g;
  }
  __syncthreads();
  C2* s = fft_lines(r, o, F2, BL, tw, true);
  for (int idx = threadIdx.x; idx < BL * N2; idx += blockDim.x) {
    const int j = idx / BL, l = idx - j * BL;
    if (kx0 + l < Hx) col0[l + zs * j] = s[l * F2 + j];
  }
}

template <typename T, typename C2>
__global__ void __launch_bounds__(kThreads) k_fft_x_inv(const C2* __restrict__ cb, T* __restrict__ U, int N0, int N1,
                                                       int N2, int F0, int F1, int BL, const C2* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  C2* y = x + BL * F0;
  const int64_t nlines = (int64_t)N1 * N2;
  const int64_t L0 = (int64_t)blockIdx.x * BL;
  const int Hx = F0 / 2 + 1;
  for (int idx = threadIdx.x; idx < BL * F0; idx += blockDim.x) {
    const int l = idx / F0, j = idx - l * F0;
    const int64_t L = L0 + l;
    C2 v = {0, 0};
    if (L < nlines) {
      const int64_t yy = L % N1, zz = L / N1;
      const C2* row = cb + (int64_t)Hx * (yy + (int64_t)F1 * zz);
      if (j < Hx) {
        v = row[j];
      } else {
        v = row[F0 - j];
        v.y = -v.y;
      }
    }
    x[idx] = v;
  }
  __syncthreads();
  C2* r = fft_lines(x, y, F0, BL, tw, true);
  for (int idx = threadIdx.x; idx < BL * N0; idx += blockDim.x) {
    const int l = idx / N0, j = idx - l * N0;
    const int64_t L = L0 + l;
    if (L < nlines) U[j + (int64_t)N0 * L] = r[l * F0 + j].x;
  }
}

template <typename C2>
int lines_per_block(int F) {
  int bl = kSmemBudget / (2 * F * (int)sizeof(C2));
  int p = 1;
  while (p * 2 <= bl && p * 2 <= 32) p *= 2;
  return p;
}

template <typename K>
void allow_smem(K kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
}

}  // namespace

template <typename T>
void launch_fft_conv(const DevOps<T>& d, cudaStream_t st) {
  using C2 = typename Vec2<T>::type;
  static bool attr_done = false;
  if (!attr_done) {
    allow_smem(k_fft_x_fwd<T, C2>);
    allow_smem(k_fft_y<C2>);
    allow_smem(k_fft_z_conv<T, C2>);
    allow_smem(k_fft_x_inv<T, C2>);
    attr_done = true;
  }
  const int N0 = d.dims[0], N1 = d.dims[1], N2 = d.dims[2];
  const int F0 = d.fft[0], F1 = d.fft[1], F2 = d.fft[2];
  const int Hx = F0 / 2 + 1;
  // 1. x forward
  {
    d.prof.begin(KID_FFT_X_FWD, st);
    const int BL = lines_per_block<C2>(F0);
    const int64_t nl = (int64_t)N1 * N2;
    k_fft_x_fwd<T, C2><<<(unsigned)((nl + BL - 1) / BL), kThreads, 2 * BL * F0 * sizeof(C2), st>>>(
        d.grid, d.cbuf, N0, N1, N2, F0, F1, BL, d.tw[0]);
    d.prof.end(KID_FFT_X_FWD, st);
  }
  // 2. y forward on the populated planes
  {
    d.prof.begin(KID_FFT_Y_FWD, st);
    const int BL = lines_per_block<C2>(F1);
    const unsigned nb = (unsigned)(((Hx + BL - 1) / BL) * N2);
    k_fft_y<C2><<<nb, kThreads, 2 * BL * F1 * sizeof(C2), st>>>(d.cbuf, Hx, F1, N2, N1, F1, BL, false, d.tw[1]);
    d.prof.end(KID_FFT_Y_FWD, st);
  }
  // 3. z forward, spectral multiply, z inverse
  {
    d.prof.begin(KID_FFT_Z_CONV, st);
    const int BL = lines_per_block<C2>(F2);
    const unsigned nb = (unsigned)(((Hx + BL - 1) / BL) * F1);
    k_fft_z_conv<T, C2><<<nb, kThreads, 2 * BL * F2 * sizeof(C2), st>>>(d.cbuf, Hx, F1, F2, N2, BL, d.ghat, d.tw[2]);
    d.prof.end(KID_FFT_Z_CONV, st);
  }
  // 4. y inverse, keep y < N1
  {
    d.prof.begin(KID_FFT_Y_INV, st);
    const int BL = lines_per_block<C2>(F1);
    const unsigned nb = (unsigned)(((Hx + BL - 1) / BL) * N2);
    k_fft_y<C2><<<nb, kThreads, 2 * BL * F1 * sizeof(C2), st>>>(d.cbuf, Hx, F1, N2, F1, N1, BL, true, d.tw[1]);
    d.prof.end(KID_FFT_Y_INV, st);
  }
  // 5. x inverse (complex to real) into the grid buffer
  {
    d.prof.begin(KID_FFT_X_INV, st);
    const int BL = lines_per_block<C2>(F0);
    const int64_t nl = (int64_t)N1 * N2;
    k_fft_x_inv<T, C2><<<(unsigned)((nl + BL - 1) / BL), kThreads, 2 * BL * F0 * sizeof(C2), st>>>(
        d.cbuf, d.grid, N0, N1, N2, F0, F1, BL, d.tw[0]);
    d.prof.end(KID_FFT_X_INV, st);
  }
}

template void launch_fft_conv<double>(const DevOps<double>&, cudaStream_t);
template void launch_fft_conv<float>(const DevOps<float>&, cudaStream_t);

}  // namespace pmfem
