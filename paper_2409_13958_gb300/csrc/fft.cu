// BAIM step 2 on sm_103a: U = IFFT( Ghat . FFT(Q) ) over the grid of Eq. 16.
// Periodic axes are transformed circularly at their own length; open axes are zero-padded
// to twice their length (linear convolution), and zero inputs are never read.  Five passes
// over a complex half-spectrum buffer laid out [z][y][kx] (kx = 0..F0/2):
//   1. x: real-to-complex on the N1 x N2 populated rows (inputs beyond N0 are zero)
//   2. y: forward on the populated z planes (inputs beyond N1 are zero)
//   3. z: forward (inputs beyond N2 zero), multiply by the real PGF spectrum, inverse,
//         keep z < N2 -- one kernel, the spectrum never leaves registers
//   4. y: inverse on the populated z planes, keep y < N1
//   5. x: complex-to-real on the kept rows, keep x < N0
//
// Line transform of length F = R1 * R2 (R1 >= R2, powers of two), two-factor form:
//   forward  X[k1 + R1 k2] = sum_n2 W_R2^{n2 k2} W_F^{n2 k1} sum_n1 x[R2 n1 + n2] W_R1^{n1 k1}
//   inverse  y[a + R2 b]   = sum_k1 W_R1^{-b k1} W_F^{-a k1} sum_k2 X[k1 + R1 k2] W_R2^{-a k2}
// Every small DFT runs on a register array (radix-2, fully unrolled); the single
// transpose between the two factors goes through padded shared memory.  A block holds
// LB lines; in strided passes consecutive threads take consecutive lines (adjacent kx),
// so each global access of a warp is one contiguous segment.
#include <mutex>
#include <set>
#include <utility>

#include "bloch.hpp"
#include "device.hpp"

namespace pmfem {
namespace {

// Register caps of the strided passes (resident blocks per SM asked of the z and the y
// passes; 0 or unset: the compiler chooses).  The passes are not DRAM-bound (the spectrum
// buffer stays in L2); ncu shows them limited by occupancy.  Measured on the 256^3 transform:
// z pass with 4 blocks per SM (128 registers instead of 139, 4 bytes of spill) 50.3 -> 47.1 us;
// 5 blocks spill 80 bytes and gain nothing; capping the y passes (3 blocks) gains nothing.
#ifndef PMFEM_FFT_Z_MINB
#define PMFEM_FFT_Z_MINB 4
#endif
#if PMFEM_FFT_Z_MINB > 0
#define PMFEM_FFT_Z_LB(n) __launch_bounds__(n, PMFEM_FFT_Z_MINB)
#else
#define PMFEM_FFT_Z_LB(n) __launch_bounds__(n)
#endif
#ifdef PMFEM_FFT_Y_MINB
#define PMFEM_FFT_Y_LB(n) __launch_bounds__(n, PMFEM_FFT_Y_MINB)
#else
#define PMFEM_FFT_Y_LB(n) __launch_bounds__(n)
#endif

template <typename C2> __device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.x + b.x, a.y + b.y}; }
template <typename C2> __device__ __forceinline__ C2 csub(C2 a, C2 b) { return {a.x - b.x, a.y - b.y}; }
template <typename C2> __device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C2> __device__ __forceinline__ C2 conjif(C2 w, bool inv) {
  if (inv) w.y = -w.y;
  return w;
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// bit-reversal permutation with compile-time indices (keeps the array in registers)
template <int R, int I, typename C2>
__device__ __forceinline__ void swap_rev(C2 (&v)[R]) {
  constexpr int J = bitrev(I, ilog2(R));
  if constexpr (J > I) {
    C2 t = v[I];
    v[I] = v[J];
    v[J] = t;
  }
}
template <int R, typename C2, int... I>
__device__ __forceinline__ void bit_reverse(C2 (&v)[R], std::integer_sequence<int, I...>) {
  (swap_rev<R, I>(v), ...);
}

// radix-2 butterfly stages of length LEN, 2 LEN, ..., R (compile-time recursion)
template <int R, int LEN, typename C2>
__device__ __forceinline__ void dft_stages(C2 (&v)[R], const C2* __restrict__ tw, int step, bool inv) {
  if constexpr (LEN <= R) {
    constexpr int half = LEN / 2;
#pragma unroll
    for (int i = 0; i < R; i += LEN) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        C2 u = v[i + k], t = v[i + k + half];
        if (k != 0) t = cmul(t, conjif(__ldg(&tw[k * (R / LEN) * step]), inv));
        v[i + k] = cadd(u, t);
        v[i + k + half] = csub(u, t);
      }
    }
    dft_stages<R, 2 * LEN>(v, tw, step, inv);
  }
}

// In-register DFT of size R, natural order in and out.  tw holds exp(-2 pi i j / F) for
// j < F and step = F / R, so W_R^j = tw[j * step].
template <int R, typename C2>
__device__ __forceinline__ void dft(C2 (&v)[R], const C2* __restrict__ tw, int step, bool inv) {
  bit_reverse<R>(v, std::make_integer_sequence<int, R>{});
  dft_stages<R, 2>(v, tw, step, inv);
}

// line geometry shared by the passes
template <int F_> struct Fac {
  static constexpr int F = F_;
  static constexpr int R1 = 1 << ((ilog2(F_) + 1) / 2);
  static constexpr int R2 = F_ / R1;
  static constexpr int IPT = R1 / R2;           // step-2 items per thread (1 or 2)
  static constexpr int LS = R1 * (R2 + 1) + 1;  // padded shared-memory line stride
};

// Forward transform of the LB lines a block holds.  ld(l, idx) returns element idx of
// line l (zero outside the populated range).  On return thread (l, j) holds, for items
// i < IPT with k1 = j + R2 i, X[k1 + R1 k2] in out[i][k2].
template <int F, int LB, bool LINE_FAST, typename C2, typename Load>
__device__ __forceinline__ void line_forward(C2* S, const C2* __restrict__ tw, Load ld, int l, int j,
                                             C2 (&out)[Fac<F>::IPT][Fac<F>::R2]) {
  using FF = Fac<F>;
  C2 a[FF::R1];
#pragma unroll
  for (int n1 = 0; n1 < FF::R1; ++n1) a[n1] = ld(l, FF::R2 * n1 + j);
  dft<FF::R1>(a, tw, FF::R2, false);
#pragma unroll
  for (int k1 = 1; k1 < FF::R1; ++k1) a[k1] = cmul(a[k1], __ldg(&tw[j * k1]));
  C2* Sl = S + l * FF::LS;
#pragma unroll
  for (int k1 = 0; k1 < FF::R1; ++k1) Sl[k1 * (FF::R2 + 1) + j] = a[k1];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < FF::IPT; ++i) {
    const int k1 = j + FF::R2 * i;
#pragma unroll
    for (int n2 = 0; n2 < FF::R2; ++n2) out[i][n2] = Sl[k1 * (FF::R2 + 1) + n2];
    dft<FF::R2>(out[i], tw, FF::R1, false);
  }
}

// Inverse transform from the layout line_forward leaves; st(l, idx, value) stores
// element idx of the result.  Unnormalised.
template <int F, int LB, bool LINE_FAST, typename C2, typename Store>
__device__ __forceinline__ void line_inverse(C2* S, const C2* __restrict__ tw, Store st, int l, int j,
                                             C2 (&in)[Fac<F>::IPT][Fac<F>::R2]) {
  using FF = Fac<F>;
  C2* Sl = S + l * FF::LS;
  __syncthreads();   // S may still be read by the forward step of another thread
#pragma unroll
  for (int i = 0; i < FF::IPT; ++i) {
    const int k1 = j + FF::R2 * i;
    dft<FF::R2>(in[i], tw, FF::R1, true);
#pragma unroll
    for (int a = 0; a < FF::R2; ++a) {
      C2 z = in[i][a];
      if (a != 0 && k1 != 0) z = cmul(z, conjif(__ldg(&tw[a * k1]), true));
      Sl[k1 * (FF::R2 + 1) + a] = z;
    }
  }
  __syncthreads();
  C2 c[FF::R1];
#pragma unroll
  for (int k1 = 0; k1 < FF::R1; ++k1) c[k1] = Sl[k1 * (FF::R2 + 1) + j];
  dft<FF::R1>(c, tw, FF::R2, true);
#pragma unroll
  for (int b = 0; b < FF::R1; ++b) st(l, j + FF::R2 * b, c[b]);
}

template <bool LINE_FAST, int LB, int R2>
__device__ __forceinline__ void thread_line(int& l, int& j) {
  const int t = threadIdx.x;
  if (LINE_FAST) {
    l = t % LB;
    j = t / LB;
  } else {
    l = t / R2;
    j = t % R2;
  }
}

// Line of a strided pass (y or z): blocks cover the columns kx in groups of LB lines per outer
// index o (o = z for the y pass, ky for the z pass).  With SPLIT, when Hx - 1 is a multiple of
// LB, the last column kx = Hx - 1 (the Nyquist column of the real-to-complex x transform) gets
// its own blocks, whose LB lines are LB consecutive outer indices, instead of one block per
// outer index with a single busy line.  Measured on the 256^3 FFT: the z pass gains (64 -> 62
// us); the y passes lose (their Nyquist lines are then a plane apart), so they keep one block
// per outer index.
template <bool SPLIT>
__device__ __forceinline__ void strided_line(int Hx, int LB, int nouter, int l, int& kx, int& o, bool& ok) {
  const int nfull = (Hx - 1) / LB;
  if (SPLIT && (Hx - 1) % LB == 0 && nfull > 0) {
    const int nb_full = nfull * nouter;
    if ((int)blockIdx.x < nb_full) {
      o = blockIdx.x / nfull;
      kx = (blockIdx.x - o * nfull) * LB + l;
      ok = true;
    } else {
      kx = Hx - 1;
      o = (blockIdx.x - nb_full) * LB + l;
      ok = o < nouter;
    }
    return;
  }
  const int kxb = (Hx + LB - 1) / LB;
  o = blockIdx.x / kxb;
  kx = (blockIdx.x - o * kxb) * LB + l;
  ok = kx < Hx;
}

template <bool SPLIT>
__host__ __forceinline__ unsigned strided_blocks(int Hx, int LB, int nouter) {
  const int nfull = (Hx - 1) / LB;
  if (SPLIT && (Hx - 1) % LB == 0 && nfull > 0) return (unsigned)(nfull * nouter + (nouter + LB - 1) / LB);
  return (unsigned)(((Hx + LB - 1) / LB) * nouter);
}

// ---------------------------------------------------------------- pass 1: x forward
template <typename T, typename C2, int F, int LB>
__global__ void __launch_bounds__(LB * Fac<F>::R2) k_fft_x_fwd(const T* __restrict__ Q, C2* __restrict__ cb, int N0,
                                                             int N1, int N2, int F1, const C2* __restrict__ tw,
                                                             const int64_t* __restrict__ boff) {
  using FF = Fac<F>;
  pdl_enter();
  if (boff) {   // batched: blockIdx.y selects the mesh, boff its (grid, spectrum buffer) offsets
    Q += boff[3 * blockIdx.y];
    cb += boff[3 * blockIdx.y + 1];
  }
  extern __shared__ unsigned char smem_raw[];
  C2* S = reinterpret_cast<C2*>(smem_raw);
  int l, j;
  thread_line<false, LB, FF::R2>(l, j);
  const int64_t nlines = (int64_t)N1 * N2;
  const int64_t L = (int64_t)blockIdx.x * LB + l;
  const bool ok = L < nlines;
  const T* row = Q + (int64_t)N0 * (ok ? L : 0);
  auto ld = [&](int, int idx) -> C2 {
    T v = (ok && idx < N0) ? row[idx] : T(0);
    return C2{v, T(0)};
  };
  C2 X[FF::IPT][FF::R2];
  line_forward<F, LB, false>(S, tw, ld, l, j, X);
  if (!ok) return;
  const int Hx = F / 2 + 1;
  const int64_t yy = L % N1, zz = L / N1;
  C2* out = cb + (int64_t)Hx * (yy + (int64_t)F1 * zz);
#pragma unroll
  for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
    for (int k2 = 0; k2 < FF::R2; ++k2) {
      const int k = j + FF::R2 * i + FF::R1 * k2;
      if (k < Hx) out[k] = X[i][k2];
    }
}

// ---------------------------------------------------------------- passes 2, 4: y
template <typename C2, int F, int LB, bool INV>
__global__ void PMFEM_FFT_Y_LB(LB * Fac<F>::R2) k_fft_y(C2* __restrict__ cb, int Hx, int n_in, int n_out,
                                                         const C2* __restrict__ tw, const int64_t* __restrict__ boff,
                                                         int nz) {
  using FF = Fac<F>;
  pdl_enter();
  if (boff) cb += boff[3 * blockIdx.y + 1];
  extern __shared__ unsigned char smem_raw[];
  C2* S = reinterpret_cast<C2*>(smem_raw);
  int l, j;
  thread_line<true, LB, FF::R2>(l, j);
  int kx, z;
  bool ok;
  strided_line<false>(Hx, LB, nz, l, kx, z, ok);
  C2* col = cb + (ok ? (int64_t)Hx * F * z + kx : 0);
  C2 X[FF::IPT][FF::R2];
  if (!INV) {
    auto ld = [&](int, int idx) -> C2 { return (ok && idx < n_in) ? col[(int64_t)Hx * idx] : C2{0, 0}; };
    line_forward<F, LB, true>(S, tw, ld, l, j, X);
    if (!ok) return;
#pragma unroll
    for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
      for (int k2 = 0; k2 < FF::R2; ++k2) col[(int64_t)Hx * (j + FF::R2 * i + FF::R1 * k2)] = X[i][k2];
  } else {
    // the inverse starts from the k1 + R1 k2 layout: load it directly
#pragma unroll
    for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
      for (int k2 = 0; k2 < FF::R2; ++k2)
        X[i][k2] = ok ? col[(int64_t)Hx * (j + FF::R2 * i + FF::R1 * k2)] : C2{0, 0};
    auto st = [&](int, int idx, C2 v) {
      if (ok && idx < n_out) col[(int64_t)Hx * idx] = v;
    };
    line_inverse<F, LB, true>(S, tw, st, l, j, X);
  }
}

// ---------------------------------------------------------------- pass 3: z convolution
// FULL: the spectrum is the full F0 x F1 x F2 grid (x fastest, Hx = F0 columns), as for the
// twisted Bloch kernel, which is real but not even; otherwise the PGF spectrum reduced by symmetry.
template <typename T, typename C2, int F, int LB, bool FULL = false>
__global__ void PMFEM_FFT_Z_LB(LB * Fac<F>::R2) k_fft_z_conv(C2* __restrict__ cb, int Hx, int F1, int N2,
                                                              const T* __restrict__ ghat, const C2* __restrict__ tw,
                                                              const int64_t* __restrict__ boff) {
  using FF = Fac<F>;
  pdl_enter();
  if (boff) {
    cb += boff[3 * blockIdx.y + 1];
    ghat += boff[3 * blockIdx.y + 2];
  }
  extern __shared__ unsigned char smem_raw[];
  C2* S = reinterpret_cast<C2*>(smem_raw);
  int l, j;
  thread_line<true, LB, FF::R2>(l, j);
  int kx, ky;
  bool ok;
  strided_line<!FULL>(Hx, LB, F1, l, kx, ky, ok);
  if (!ok) kx = 0, ky = 0;
  const int64_t zs = (int64_t)Hx * F1;
  C2* col = cb + (int64_t)Hx * ky + kx;
  auto ld = [&](int, int idx) -> C2 { return (ok && idx < N2) ? col[zs * idx] : C2{0, 0}; };
  C2 X[FF::IPT][FF::R2];
  line_forward<F, LB, true>(S, tw, ld, l, j, X);
  // spectral multiply by the real PGF spectrum (reduced by symmetry in every axis unless FULL)
  const int H1 = F1 / 2 + 1;
  const int iy = FULL ? ky : (ky <= F1 - ky ? ky : F1 - ky);
  const T* g = ghat + (ok ? kx : 0) + (int64_t)Hx * iy;
  const int64_t gs = (int64_t)Hx * (FULL ? F1 : H1);
#pragma unroll
  for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
    for (int k2 = 0; k2 < FF::R2; ++k2) {
      const int kz = j + FF::R2 * i + FF::R1 * k2;
      const int iz = FULL ? kz : (kz <= F - kz ? kz : F - kz);
      const T gv = ok ? __ldg(&g[gs * iz]) : T(0);
      X[i][k2].x *= gv;
      X[i][k2].y *= gv;
    }
  auto st = [&](int, int idx, C2 v) {
    if (ok && idx < N2) col[zs * idx] = v;
  };
  line_inverse<F, LB, true>(S, tw, st, l, j, X);
}

// ---------------------------------------------------------------- pass 5: x inverse (C2R)
template <typename T, typename C2, int F, int LB>
__global__ void __launch_bounds__(LB * Fac<F>::R2) k_fft_x_inv(const C2* __restrict__ cb, T* __restrict__ U, int N0,
                                                             int N1, int N2, int F1, const C2* __restrict__ tw,
                                                             const int64_t* __restrict__ boff) {
  using FF = Fac<F>;
  pdl_enter();
  if (boff) {
    U += boff[3 * blockIdx.y];
    cb += boff[3 * blockIdx.y + 1];
  }
  extern __shared__ unsigned char smem_raw[];
  C2* S = reinterpret_cast<C2*>(smem_raw);
  int l, j;
  thread_line<false, LB, FF::R2>(l, j);
  const int64_t nlines = (int64_t)N1 * N2;
  const int64_t L = (int64_t)blockIdx.x * LB + l;
  const bool ok = L < nlines;
  const int Hx = F / 2 + 1;
  const int64_t yy = ok ? L % N1 : 0, zz = ok ? L / N1 : 0;
  const C2* row = cb + (int64_t)Hx * (yy + (int64_t)F1 * zz);
  C2 X[FF::IPT][FF::R2];
#pragma unroll
  for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
    for (int k2 = 0; k2 < FF::R2; ++k2) {
      const int k = j + FF::R2 * i + FF::R1 * k2;
      C2 v = {0, 0};
      if (ok) {
        if (k < Hx) {
          v = row[k];
        } else {
          v = row[F - k];   // Hermitian symmetry of a real signal
          v.y = -v.y;
        }
      }
      X[i][k2] = v;
    }
  T* out = U + (int64_t)N0 * (ok ? L : 0);
  auto st = [&](int, int idx, C2 v) {
    if (ok && idx < N0) out[idx] = v.x;
  };
  line_inverse<F, LB, false>(S, tw, st, l, j, X);
}

// ---------------------------------------------------------------- complex x lines
// Lines along x of a complex grid (the Bloch convolution and the FP64 transform of its kernel
// table): line L = y + ny z reads src[ss_y y + ss_z z + idx] for idx < n_in (zero beyond) and
// writes dst[ds_y y + ds_z z + k] for k < n_out, times scale; forward, or inverse (INV).  src may
// be dst when the strides agree: a line is read whole before any of it is written.
template <typename C2, int F, int LB, bool INV>
__global__ void __launch_bounds__(LB * Fac<F>::R2) k_cfft_x(const C2* src, C2* dst, int ny, int nz, int64_t ss_y,
                                                          int64_t ss_z, int64_t ds_y, int64_t ds_z, int n_in,
                                                          int n_out, double scale, const C2* __restrict__ tw) {
  using FF = Fac<F>;
  using E = decltype(C2::x);
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  C2* S = reinterpret_cast<C2*>(smem_raw);
  int l, j;
  thread_line<false, LB, FF::R2>(l, j);
  const int64_t L = (int64_t)blockIdx.x * LB + l;
  const bool ok = L < (int64_t)ny * nz;
  const int64_t yy = ok ? L % ny : 0, zz = ok ? L / ny : 0;
  const C2* in = src + ss_y * yy + ss_z * zz;
  C2* out = dst + ds_y * yy + ds_z * zz;
  const E sc = (E)scale;
  C2 X[FF::IPT][FF::R2];
  if (!INV) {
    auto ld = [&](int, int idx) -> C2 { return (ok && idx < n_in) ? in[idx] : C2{0, 0}; };
    line_forward<F, LB, false>(S, tw, ld, l, j, X);
    if (!ok) return;
#pragma unroll
    for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
      for (int k2 = 0; k2 < FF::R2; ++k2) {
        const int k = j + FF::R2 * i + FF::R1 * k2;
        if (k < n_out) out[k] = C2{X[i][k2].x * sc, X[i][k2].y * sc};
      }
  } else {
#pragma unroll
    for (int i = 0; i < FF::IPT; ++i)
#pragma unroll
      for (int k2 = 0; k2 < FF::R2; ++k2) {
        const int k = j + FF::R2 * i + FF::R1 * k2;
        X[i][k2] = (ok && k < n_in) ? in[k] : C2{0, 0};
      }
    auto st = [&](int, int idx, C2 v) {
      if (ok && idx < n_out) out[idx] = C2{v.x * sc, v.y * sc};
    };
    line_inverse<F, LB, false>(S, tw, st, l, j, X);
  }
}

// Line counts per block (measured on the 256^3 transform of the 1M-node wire): the y passes
// read 128-byte rows of 16 adjacent FP32 lines; the z pass, whose block also multiplies by the
// spectrum and transforms back, runs faster with 8 lines (more blocks in flight); the
// contiguous x passes take 128 threads per block.  FP64 halves the strided line counts.
#ifndef PMFEM_FFT_LBS
#define PMFEM_FFT_LBS 16
#endif
#ifndef PMFEM_FFT_LBZ
#define PMFEM_FFT_LBZ 8
#endif
#ifndef PMFEM_FFT_TPB
#define PMFEM_FFT_TPB 128
#endif
template <typename T> struct Lines {
  static constexpr int STRIDED = sizeof(T) == 4 ? PMFEM_FFT_LBS : PMFEM_FFT_LBS / 2;
  static constexpr int Z = sizeof(T) == 4 ? PMFEM_FFT_LBZ : (PMFEM_FFT_LBZ / 2 > 0 ? PMFEM_FFT_LBZ / 2 : 1);
};

template <typename T, int F>
struct Passes {
  using C2 = typename Vec2<T>::type;
  using FF = Fac<F>;
  static constexpr int LBX = (PMFEM_FFT_TPB / FF::R2) > 0 ? (PMFEM_FFT_TPB / FF::R2) : 1;   // contiguous passes
  static constexpr int LBS = Lines<T>::STRIDED;
  static constexpr int LBZ = Lines<T>::Z;
  static size_t smem(int lb) { return (size_t)lb * FF::LS * sizeof(C2); }

  static void x_fwd(const FftArgs<T>& d, cudaStream_t st) {
    const int64_t nl = (int64_t)d.dims[1] * d.dims[2];
    const size_t sm = smem(LBX);
    set_smem(k_fft_x_fwd<T, C2, F, LBX>, sm);
    launch_k(k_fft_x_fwd<T, C2, F, LBX>, dim3((unsigned)((nl + LBX - 1) / LBX), d.count), LBX * FF::R2, sm, st,
        d.grid, d.cbuf, d.dims[0], d.dims[1], d.dims[2], d.fft[1], d.tw[0], d.boff);
  }
  static void x_inv(const FftArgs<T>& d, cudaStream_t st) {
    const int64_t nl = (int64_t)d.dims[1] * d.dims[2];
    const size_t sm = smem(LBX);
    set_smem(k_fft_x_inv<T, C2, F, LBX>, sm);
    launch_k(k_fft_x_inv<T, C2, F, LBX>, dim3((unsigned)((nl + LBX - 1) / LBX), d.count), LBX * FF::R2, sm, st,
        d.cbuf, d.grid, d.dims[0], d.dims[1], d.dims[2], d.fft[1], d.tw[0], d.boff);
  }
  static void y(const FftArgs<T>& d, bool inv, cudaStream_t st) {
    const int Hx = d.fft[0] / 2 + 1;
    const unsigned nb = strided_blocks<false>(Hx, LBS, d.dims[2]);
    const size_t sm = smem(LBS);
    if (!inv) {
      set_smem(k_fft_y<C2, F, LBS, false>, sm);
      launch_k(k_fft_y<C2, F, LBS, false>, dim3(nb, d.count), LBS * FF::R2, sm, st, d.cbuf, Hx, d.dims[1], F, d.tw[1],
                                                                               d.boff, d.dims[2]);
    } else {
      set_smem(k_fft_y<C2, F, LBS, true>, sm);
      launch_k(k_fft_y<C2, F, LBS, true>, dim3(nb, d.count), LBS * FF::R2, sm, st, d.cbuf, Hx, F, d.dims[1], d.tw[1],
                                                                              d.boff, d.dims[2]);
    }
  }
  // complex lines along x (k_cfft_x)
  static void cx(const C2* src, C2* dst, int ny, int nz, int64_t ssy, int64_t ssz, int64_t dsy, int64_t dsz, int n_in,
                 int n_out, double scale, bool inv, const C2* tw, cudaStream_t st) {
    const int64_t nl = (int64_t)ny * nz;
    const dim3 grid((unsigned)((nl + LBX - 1) / LBX));
    const size_t sm = smem(LBX);
    if (!inv) {
      set_smem(k_cfft_x<C2, F, LBX, false>, sm);
      launch_k(k_cfft_x<C2, F, LBX, false>, grid, LBX * FF::R2, sm, st, src, dst, ny, nz, ssy, ssz, dsy, dsz, n_in,
               n_out, scale, tw);
    } else {
      set_smem(k_cfft_x<C2, F, LBX, true>, sm);
      launch_k(k_cfft_x<C2, F, LBX, true>, grid, LBX * FF::R2, sm, st, src, dst, ny, nz, ssy, ssz, dsy, dsz, n_in,
               n_out, scale, tw);
    }
  }
  // strided lines of length F over Hx adjacent columns in each of nz planes (plane stride Hx F):
  // the y pass of a complex grid, or the z pass of a whole grid as Hx = F0 F1, nz = 1
  static void cy(C2* cb, int Hx, int n_in, int n_out, int nz, bool inv, const C2* tw, cudaStream_t st) {
    const unsigned nb = strided_blocks<false>(Hx, LBS, nz);
    const size_t sm = smem(LBS);
    if (!inv) {
      set_smem(k_fft_y<C2, F, LBS, false>, sm);
      launch_k(k_fft_y<C2, F, LBS, false>, dim3(nb), LBS * FF::R2, sm, st, cb, Hx, n_in, n_out, tw,
               (const int64_t*)nullptr, nz);
    } else {
      set_smem(k_fft_y<C2, F, LBS, true>, sm);
      launch_k(k_fft_y<C2, F, LBS, true>, dim3(nb), LBS * FF::R2, sm, st, cb, Hx, n_in, n_out, tw,
               (const int64_t*)nullptr, nz);
    }
  }
  // z forward, multiply by the full real spectrum, z inverse, on the Hx = F0 columns of F1 rows
  static void cz_conv(C2* cb, int F0, int F1, int N2, const T* spec, const C2* tw, cudaStream_t st) {
    const unsigned nb = strided_blocks<false>(F0, LBZ, F1);
    const size_t sm = smem(LBZ);
    set_smem(k_fft_z_conv<T, C2, F, LBZ, true>, sm);
    launch_k(k_fft_z_conv<T, C2, F, LBZ, true>, dim3(nb), LBZ * FF::R2, sm, st, cb, F0, F1, N2, spec, tw,
             (const int64_t*)nullptr);
  }
  static void z(const FftArgs<T>& d, cudaStream_t st) {
    const int Hx = d.fft[0] / 2 + 1;
    const unsigned nb = strided_blocks<true>(Hx, LBZ, d.fft[1]);
    const size_t sm = smem(LBZ);
    set_smem(k_fft_z_conv<T, C2, F, LBZ>, sm);
    launch_k(k_fft_z_conv<T, C2, F, LBZ>, dim3(nb, d.count), LBZ * FF::R2, sm, st, d.cbuf, Hx, d.fft[1], d.dims[2],
                                                                             d.ghat, d.tw[2], d.boff);
  }
};

#define PMFEM_FFT_DISPATCH(F, CALL)                     \
  switch (F) {                                          \
    case 4: Passes<T, 4>::CALL; break;                  \
    case 8: Passes<T, 8>::CALL; break;                  \
    case 16: Passes<T, 16>::CALL; break;                \
    case 32: Passes<T, 32>::CALL; break;                \
    case 64: Passes<T, 64>::CALL; break;                \
    case 128: Passes<T, 128>::CALL; break;              \
    case 256: Passes<T, 256>::CALL; break;              \
    case 512: Passes<T, 512>::CALL; break;              \
    default: Passes<T, 1024>::CALL; break;              \
  }

}  // namespace

template <typename T>
void launch_fft(const FftArgs<T>& a, const ProfHook& prof, cudaStream_t st) {
  prof.begin(KID_FFT_X_FWD, st);
  PMFEM_FFT_DISPATCH(a.fft[0], x_fwd(a, st));
  prof.end(KID_FFT_X_FWD, st);
  prof.begin(KID_FFT_Y_FWD, st);
  PMFEM_FFT_DISPATCH(a.fft[1], y(a, false, st));
  prof.end(KID_FFT_Y_FWD, st);
  prof.begin(KID_FFT_Z_CONV, st);
  PMFEM_FFT_DISPATCH(a.fft[2], z(a, st));
  prof.end(KID_FFT_Z_CONV, st);
  prof.begin(KID_FFT_Y_INV, st);
  PMFEM_FFT_DISPATCH(a.fft[1], y(a, true, st));
  prof.end(KID_FFT_Y_INV, st);
  prof.begin(KID_FFT_X_INV, st);
  PMFEM_FFT_DISPATCH(a.fft[0], x_inv(a, st));
  prof.end(KID_FFT_X_INV, st);
}

template <typename T>
void launch_fft_conv(const DevOps<T>& d, cudaStream_t st) {
  FftArgs<T> a;
  a.grid = d.grid;
  a.cbuf = d.cbuf;
  a.ghat = d.ghat;
  for (int k = 0; k < 3; ++k) {
    a.dims[k] = d.dims[k];
    a.fft[k] = d.fft[k];
    a.tw[k] = d.tw[k];
  }
  launch_fft(a, d.prof, st);
}

template <typename T, typename C2>
void launch_bloch_fft_conv(const C2* Q, C2* U, C2* cb, const T* spec, const int dims[3], const int fft[3],
                           const C2* const tw[3], cudaStream_t st) {
  const int N0 = dims[0], N1 = dims[1], N2 = dims[2];
  const int F0 = fft[0], F1 = fft[1], F2 = fft[2];
  const int64_t row = F0, plane = (int64_t)F0 * F1;
  // 1. x forward on the populated rows (y < N1, z < N2), inputs beyond N0 zero
  PMFEM_FFT_DISPATCH(F0, cx(Q, cb, N1, N2, N0, (int64_t)N0 * N1, row, plane, N0, F0, 1.0, false, tw[0], st));
  // 2. y forward on the populated planes (inputs beyond N1 zero)
  PMFEM_FFT_DISPATCH(F1, cy(cb, F0, N1, F1, N2, false, tw[1], st));
  // 3. z forward (inputs beyond N2 zero), times the spectrum, z inverse, keep z < N2
  PMFEM_FFT_DISPATCH(F2, cz_conv(cb, F0, F1, N2, spec, tw[2], st));
  // 4. y inverse on the kept planes, keep y < N1
  PMFEM_FFT_DISPATCH(F1, cy(cb, F0, F1, N1, N2, true, tw[1], st));
  // 5. x inverse on the kept rows, keep x < N0, scaled by 1 / (F0 F1 F2)
  PMFEM_FFT_DISPATCH(F0, cx(cb, U, N1, N2, row, plane, N0, (int64_t)N0 * N1, F0, N0,
                            1.0 / ((double)F0 * F1 * F2), true, tw[0], st));
}

void launch_fft3_forward_f64(double2* buf, const int fft[3], const double2* const tw[3], cudaStream_t st) {
  using T = double;
  const int F0 = fft[0], F1 = fft[1], F2 = fft[2];
  const int64_t plane = (int64_t)F0 * F1;
  PMFEM_FFT_DISPATCH(F0, cx(buf, buf, F1, F2, F0, plane, F0, plane, F0, F0, 1.0, false, tw[0], st));
  PMFEM_FFT_DISPATCH(F1, cy(buf, F0, F1, F1, F2, false, tw[1], st));
  PMFEM_FFT_DISPATCH(F2, cy(buf, F0 * F1, F2, F2, 1, false, tw[2], st));
}

template void launch_bloch_fft_conv<double, double2>(const double2*, double2*, double2*, const double*, const int*,
                                                     const int*, const double2* const*, cudaStream_t);
template void launch_bloch_fft_conv<float, float2>(const float2*, float2*, float2*, const float*, const int*,
                                                   const int*, const float2* const*, cudaStream_t);
template void launch_fft_conv<double>(const DevOps<double>&, cudaStream_t);
template void launch_fft_conv<float>(const DevOps<float>&, cudaStream_t);
template void launch_fft<float>(const FftArgs<float>&, const ProfHook&, cudaStream_t);

}  // namespace pmfem
