// Kernels of the implicit midpoint LLG step (Sec. 2.2: the paper integrates the discrete LLG
// system with implicit schemes solved by Newton iterations and a preconditioned Krylov solver).
// Everything here is node-local or a reduction; the only non-local operation of a step, the
// field (and, inside the Krylov solver, the field's linear part applied to a vector), is the
// library's own field evaluation.  Vectors are N' x 3 in the C-ABI unknown order.
//
//   f(m)      = -g [ m x H + alpha m x (m x H) ],  g = gamma0 / (1 + alpha^2)
//   R(y)      = y - m0 - dt f(mb),  mb = (m0 + y) / 2,  H = H(mb)
//   J v       = v - (dt/2) Df(mb) v
//   Df(m) v   = -g [ v x H + m x Av + alpha ( v x (m x H) + m x (v x H) + m x (m x Av) ) ]
//   P_n       = J restricted to node n with Av replaced by c_n v (c_n: the exchange operator's
//               own coefficient); the preconditioner applies P_n^-1 node by node.
#include <cuda_runtime.h>

#include <cstdint>

#include "implicit.hpp"

namespace pmfem {
namespace {

constexpr int kB = 256;

// Node-local arithmetic runs in the vectors' own type T (FP32 vectors: FP32 arithmetic; GB300's
// FP64 units are narrow, and at one FP64 operation per element per Gram-Schmidt coefficient the
// FP32 step spent most of its time in them); the reductions sum blocks in FP64.
template <typename C>
__device__ __forceinline__ void cross3(const C* a, const C* b, C* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ void load3(const T* p, int64_t i, T* v) {
  v[0] = p[3 * i];
  v[1] = p[3 * i + 1];
  v[2] = p[3 * i + 2];
}

// -g [ m x H + alpha m x (m x H) ]
template <typename C>
__device__ __forceinline__ void llg_f(const C* m, const C* H, C g, C alpha, C* f) {
  C mxH[3], mmH[3];
  cross3(m, H, mxH);
  cross3(m, mxH, mmH);
  for (int d = 0; d < 3; ++d) f[d] = -g * (mxH[d] + alpha * mmH[d]);
}

template <typename T>
__global__ void k_mid(int64_t n, const T* __restrict__ m0, const T* __restrict__ y, T* __restrict__ mb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  mb[i] = (T)0.5 * (m0[i] + y[i]);
}

template <typename T>
__global__ void k_residual(int64_t n, const T* __restrict__ m0, const T* __restrict__ y, const T* __restrict__ mb,
                           const T* __restrict__ H, T dt, T g, T alpha, T* __restrict__ R) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T m[3], h[3], f[3];
  load3(mb, i, m);
  load3(H, i, h);
  llg_f(m, h, g, alpha, f);
  for (int d = 0; d < 3; ++d) R[3 * i + d] = y[3 * i + d] - m0[3 * i + d] - dt * f[d];
}

// out = v - (dt/2) Df(mb) v, given Av (the field's linear part applied to v); hdg = (dt/2)(-g)
template <typename T>
__global__ void k_jvp(int64_t n, const T* __restrict__ mb, const T* __restrict__ H, const T* __restrict__ Av,
                      const T* __restrict__ v, T hdg, T alpha, T* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T m[3], h[3], a[3], x[3];
  load3(mb, i, m);
  load3(H, i, h);
  load3(Av, i, a);
  load3(v, i, x);
  T t[3], u[3], mxH[3], w[3];
  cross3(x, h, t);                 // v x H
  cross3(m, a, u);                 // m x Av
  for (int d = 0; d < 3; ++d) t[d] += u[d];
  cross3(m, h, mxH);
  cross3(x, mxH, w);               // v x (m x H)
  T s[3];
  for (int d = 0; d < 3; ++d) s[d] = w[d];
  T vxH[3];
  cross3(x, h, vxH);
  cross3(m, vxH, w);               // m x (v x H)
  for (int d = 0; d < 3; ++d) s[d] += w[d];
  cross3(m, a, u);
  cross3(m, u, w);                 // m x (m x Av)
  for (int d = 0; d < 3; ++d) s[d] += w[d];
  for (int d = 0; d < 3; ++d) out[3 * i + d] = x[d] - hdg * (t[d] + alpha * s[d]);
}

// P_n^-1 (row-major 3x3 per node) of the block-Jacobi preconditioner; hdg = (dt/2)(-g)
template <typename T>
__global__ void k_blocks(int64_t n, const T* __restrict__ mb, const T* __restrict__ H, const T* __restrict__ c,
                         T hdg, T alpha, T* __restrict__ Pinv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T m[3], h[3];
  load3(mb, i, m);
  load3(H, i, h);
  const T cn = c[i];
  T P[3][3];
  for (int col = 0; col < 3; ++col) {   // P e_col = e_col - (dt/2) (-g) [local Df] e_col
    T x[3] = {0, 0, 0};
    x[col] = 1;
    T t[3], u[3], mxH[3], w[3], s[3], vxH[3];
    cross3(x, h, t);
    cross3(m, x, u);
    for (int d = 0; d < 3; ++d) t[d] += cn * u[d];
    cross3(m, h, mxH);
    cross3(x, mxH, s);
    cross3(x, h, vxH);
    cross3(m, vxH, w);
    for (int d = 0; d < 3; ++d) s[d] += w[d];
    cross3(m, u, w);
    for (int d = 0; d < 3; ++d) s[d] += cn * w[d];
    for (int d = 0; d < 3; ++d) P[d][col] = x[d] - hdg * (t[d] + alpha * s[d]);
  }
  // inverse by the adjugate
  const T a00 = P[1][1] * P[2][2] - P[1][2] * P[2][1];
  const T a01 = P[0][2] * P[2][1] - P[0][1] * P[2][2];
  const T a02 = P[0][1] * P[1][2] - P[0][2] * P[1][1];
  const T a10 = P[1][2] * P[2][0] - P[1][0] * P[2][2];
  const T a11 = P[0][0] * P[2][2] - P[0][2] * P[2][0];
  const T a12 = P[0][2] * P[1][0] - P[0][0] * P[1][2];
  const T a20 = P[1][0] * P[2][1] - P[1][1] * P[2][0];
  const T a21 = P[0][1] * P[2][0] - P[0][0] * P[2][1];
  const T a22 = P[0][0] * P[1][1] - P[0][1] * P[1][0];
  const T det = P[0][0] * a00 + P[0][1] * a10 + P[0][2] * a20;
  const T id = (T)1 / det;
  const T inv[9] = {a00 * id, a01 * id, a02 * id, a10 * id, a11 * id, a12 * id, a20 * id, a21 * id, a22 * id};
  for (int k = 0; k < 9; ++k) Pinv[9 * i + k] = inv[k];
}

template <typename T>
__global__ void k_apply_blocks(int64_t n, const T* __restrict__ Pinv, const T* __restrict__ x, T* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T v[3];
  load3(x, i, v);
  for (int r = 0; r < 3; ++r)
    out[3 * i + r] = Pinv[9 * i + 3 * r] * v[0] + Pinv[9 * i + 3 * r + 1] * v[1] + Pinv[9 * i + 3 * r + 2] * v[2];
}

// partial[j * gridDim.x + b] = sum over block b's share of V_j . w (blockIdx.y = j): each thread
// sums its elements in T, the block combines the threads in FP64, all in a fixed order (the grid
// size is fixed), so the result does not change from run to run
template <typename T>
__global__ void k_multidot(int64_t len, VecList<T> V, const T* __restrict__ w, double* __restrict__ partial) {
  __shared__ double red[kB / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* __restrict__ v = V.p[blockIdx.y];
  T acc_t = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    acc_t += v[i] * w[i];
  double acc = (double)acc_t;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < kB / 32; ++k) s += red[k];
    partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// out[j] = sum_b partial[j * nblocks + b], one warp per j
__global__ void k_sum_partials(int nblocks, const double* __restrict__ partial, double* __restrict__ out) {
  const int j = blockIdx.x, lane = threadIdx.x;
  double s = 0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(int64_t)j * nblocks + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[j] = s;
}

// w = a w + sum_j coef[j] V_j  (coef on the device)
// w = a w + sum_j (csign coef[j]) V_j, the coefficients rounded to T once per block
template <typename T>
__global__ void k_combine(int64_t len, VecList<T> V, int cnt, const double* __restrict__ coef, double csign,
                          double a, T* __restrict__ w) {
  __shared__ T c[kMaxKrylov + 1];
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) c[j] = (T)(csign * coef[j]);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= len) return;
  T s = a == 0.0 ? (T)0 : (T)a * w[i];
  for (int j = 0; j < cnt; ++j) s += c[j] * V.p[j][i];
  w[i] = s;
}

// out = w / sqrt(*n2) (zero when *n2 is not positive); n2 is a device scalar
template <typename T>
__global__ void k_scale_invnorm(int64_t len, const T* __restrict__ w, const double* __restrict__ n2,
                                T* __restrict__ out) {
  __shared__ T inv;
  if (threadIdx.x == 0) inv = *n2 > 0 ? (T)(1.0 / sqrt(*n2)) : (T)0;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < len) out[i] = w[i] * inv;
}

unsigned blocks(int64_t n) { return (unsigned)((n + kB - 1) / kB); }

}  // namespace

template <typename T>
void imp_mid(int64_t n, const T* m0, const T* y, T* mb, cudaStream_t st) {
  k_mid<T><<<blocks(3 * n), kB, 0, st>>>(n, m0, y, mb);
}
template <typename T>
void imp_residual(int64_t n, const T* m0, const T* y, const T* mb, const T* H, double dt, double g, double alpha,
                  T* R, cudaStream_t st) {
  k_residual<T><<<blocks(n), kB, 0, st>>>(n, m0, y, mb, H, (T)dt, (T)g, (T)alpha, R);
}
template <typename T>
void imp_jvp(int64_t n, const T* mb, const T* H, const T* Av, const T* v, double dt, double g, double alpha, T* out,
             cudaStream_t st) {
  k_jvp<T><<<blocks(n), kB, 0, st>>>(n, mb, H, Av, v, (T)(0.5 * dt * (-g)), (T)alpha, out);
}
template <typename T>
void imp_blocks(int64_t n, const T* mb, const T* H, const T* c, double dt, double g, double alpha, T* Pinv,
                cudaStream_t st) {
  k_blocks<T><<<blocks(n), kB, 0, st>>>(n, mb, H, c, (T)(0.5 * dt * (-g)), (T)alpha, Pinv);
}
template <typename T>
void imp_apply_blocks(int64_t n, const T* Pinv, const T* x, T* out, cudaStream_t st) {
  k_apply_blocks<T><<<blocks(n), kB, 0, st>>>(n, Pinv, x, out);
}
template <typename T>
void imp_multidot(int64_t len, const VecList<T>& V, int cnt, const T* w, double* partial, int nblocks, double* out,
                  cudaStream_t st) {
  k_multidot<T><<<dim3(nblocks, cnt), kB, 0, st>>>(len, V, w, partial);
  k_sum_partials<<<cnt, 32, 0, st>>>(nblocks, partial, out);
}
template <typename T>
void imp_combine(int64_t len, const VecList<T>& V, int cnt, const double* coef, double csign, double a, T* w,
                 cudaStream_t st) {
  k_combine<T><<<blocks(len), kB, 0, st>>>(len, V, cnt, coef, csign, a, w);
}
template <typename T>
void imp_scale_invnorm(int64_t len, const T* w, const double* n2, T* out, cudaStream_t st) {
  k_scale_invnorm<T><<<blocks(len), kB, 0, st>>>(len, w, n2, out);
}

#define PMFEM_IMP_INST(T)                                                                                       \
  template void imp_mid<T>(int64_t, const T*, const T*, T*, cudaStream_t);                                      \
  template void imp_residual<T>(int64_t, const T*, const T*, const T*, const T*, double, double, double, T*,    \
                                cudaStream_t);                                                                  \
  template void imp_jvp<T>(int64_t, const T*, const T*, const T*, const T*, double, double, double, T*,         \
                           cudaStream_t);                                                                       \
  template void imp_blocks<T>(int64_t, const T*, const T*, const T*, double, double, double, T*, cudaStream_t); \
  template void imp_apply_blocks<T>(int64_t, const T*, const T*, T*, cudaStream_t);                             \
  template void imp_multidot<T>(int64_t, const VecList<T>&, int, const T*, double*, int, double*, cudaStream_t); \
  template void imp_combine<T>(int64_t, const VecList<T>&, int, const double*, double, double, T*, cudaStream_t); \
  template void imp_scale_invnorm<T>(int64_t, const T*, const double*, T*, cudaStream_t);
PMFEM_IMP_INST(double)
PMFEM_IMP_INST(float)
#undef PMFEM_IMP_INST

}  // namespace pmfem
