// Field-evaluation kernels for sm_103a: charges (Eq. 14a) with the touching-element part
// of Eq. 14c, projection onto the grid (BAIM step 1), interpolation plus precorrection
// (steps 3 and 4), and the gradient (Eq. 14d) + exchange (Eq. 8) pass with the fused
// RK4 stage update of the LLG equation (Eq. 2).
#include <cmath>
#include <cstdio>

#include "device.hpp"

namespace pmfem {

namespace {

constexpr int kG = 8;          // lanes cooperating on one sparse row
constexpr int kBlock = 256;

template <typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, kG);
  return v;
}

template <typename T, int P>
__device__ __forceinline__ void lagrange(T s, T (&w)[P]) {
#pragma unroll
  for (int i = 0; i < P; ++i) {
    T v = T(1);
#pragma unroll
    for (int j = 0; j < P; ++j)
      if (j != i) v *= (s - T(j)) / T(i - j);
    w[i] = v;
  }
}

__device__ __forceinline__ int wrap(int i, int N, bool per) {
  if (per) {
    if (i < 0) i += N;
    if (i >= N) i -= N;
  }
  return i;
}

// ---------------------------------------------------------------- charges
template <typename T>
__global__ void __launch_bounds__(kBlock) k_charges(int64_t Np, const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const T* __restrict__ wx,
                                                   const T* __restrict__ wy, const T* __restrict__ wz,
                                                   const T* __restrict__ ex, const T* __restrict__ ey,
                                                   const T* __restrict__ ez, const T* __restrict__ m,
                                                   T* __restrict__ q, T* __restrict__ e, int* flag) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kG;
  const int lane = threadIdx.x % kG;
  const bool valid = row < Np;
  T aq = 0, ae = 0;
  bool bad = false;
  if (valid) {
    const int32_t b = rowptr[row], en = rowptr[row + 1];
    for (int32_t p = b + lane; p < en; p += kG) {
      const int64_t k = col[p];
      const T mx = m[3 * k], my = m[3 * k + 1], mz = m[3 * k + 2];
      bad |= !(isfinite(mx) && isfinite(my) && isfinite(mz));
      aq += wx[p] * mx + wy[p] * my + wz[p] * mz;
      ae += ex[p] * mx + ey[p] * my + ez[p] * mz;
    }
  }
  aq = group_sum(aq);
  ae = group_sum(ae);
  if (valid && lane == 0) {
    q[row] = aq;
    e[row] = ae;
  }
  if (bad) atomicOr(flag, FLAG_NONFINITE_IN);
}

// ---------------------------------------------------------------- projection (step 1)
template <typename T, int P>
__global__ void __launch_bounds__(kBlock) k_anterp(int64_t Np, const int32_t* __restrict__ base,
                                                  const T* __restrict__ frac, const T* __restrict__ q,
                                                  T* __restrict__ grid, int N0, int N1, int N2, bool p0, bool p1,
                                                  bool p2) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= Np) return;
  T w0[P], w1[P], w2[P];
  lagrange<T, P>(frac[3 * n], w0);
  lagrange<T, P>(frac[3 * n + 1], w1);
  lagrange<T, P>(frac[3 * n + 2], w2);
  const int b0 = base[3 * n], b1 = base[3 * n + 1], b2 = base[3 * n + 2];
  const T qn = q[n];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int iz = wrap(b2 + k, N2, p2);
    const T wz = w2[k] * qn;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int iy = wrap(b1 + j, N1, p1);
      const T wzy = wz * w1[j];
      T* rowp = grid + (int64_t)N0 * (iy + (int64_t)N1 * iz);
#pragma unroll
      for (int i = 0; i < P; ++i) atomicAdd(rowp + wrap(b0 + i, N0, p0), wzy * w0[i]);
    }
  }
}

// ---------------------------------------------------------------- interpolation + precorrection
template <typename T, int P>
__global__ void __launch_bounds__(kBlock) k_interp(int64_t Np, const int32_t* __restrict__ base,
                                                  const T* __restrict__ frac, const T* __restrict__ U, int N0,
                                                  int N1, int N2, bool p0, bool p1, bool p2,
                                                  const int32_t* __restrict__ rowptrC, const int32_t* __restrict__ colC,
                                                  const T* __restrict__ valC, const int32_t* __restrict__ rowptrX,
                                                  const int32_t* __restrict__ colX, const T* __restrict__ valX,
                                                  const T* __restrict__ q, const T* __restrict__ e,
                                                  const T* __restrict__ m, T* __restrict__ u) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kG;
  const int lane = threadIdx.x % kG;
  const bool valid = row < Np;
  T acc = 0;
  if (valid) {
    T w0[P], w1[P], w2[P];
    lagrange<T, P>(frac[3 * row], w0);
    lagrange<T, P>(frac[3 * row + 1], w1);
    lagrange<T, P>(frac[3 * row + 2], w2);
    const int b0 = base[3 * row], b1 = base[3 * row + 1], b2 = base[3 * row + 2];
    for (int idx = lane; idx < P * P * P; idx += kG) {
      const int i = idx % P, j = (idx / P) % P, k = idx / (P * P);
      const int ix = wrap(b0 + i, N0, p0), iy = wrap(b1 + j, N1, p1), iz = wrap(b2 + k, N2, p2);
      acc += w0[i] * w1[j] * w2[k] * U[ix + (int64_t)N0 * (iy + (int64_t)N1 * iz)];
    }
    for (int32_t p = rowptrC[row] + lane; p < rowptrC[row + 1]; p += kG) acc += valC[p] * q[colC[p]];
    for (int32_t p = rowptrX[row] + lane; p < rowptrX[row + 1]; p += kG) {
      const int64_t k = colX[p];
      acc += valX[3 * p] * m[3 * k] + valX[3 * p + 1] * m[3 * k + 1] + valX[3 * p + 2] * m[3 * k + 2];
    }
  }
  acc = group_sum(acc);
  if (valid && lane == 0) u[row] = acc + e[row];
}

// ---------------------------------------------------------------- gradient + exchange + RK4
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock) k_field(int64_t Np, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ col, const T* __restrict__ gx,
                                                 const T* __restrict__ gy, const T* __restrict__ gz,
                                                 const T* __restrict__ kp, const T* __restrict__ u,
                                                 const T* __restrict__ m, T* __restrict__ H, int use_ms, int use_ex,
                                                 T hx, T hy, T hz, T* __restrict__ m0, T* __restrict__ mnext,
                                                 T* __restrict__ accb, T cdt, T bw, int acc_init, T dt6, T gam,
                                                 T alpha, int* flag) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kG;
  const int lane = threadIdx.x % kG;
  const bool valid = row < Np;
  T ax = 0, ay = 0, az = 0;
  if (valid) {
    const int32_t b = rowptr[row], en = rowptr[row + 1];
    for (int32_t p = b + lane; p < en; p += kG) {
      const int64_t k = col[p];
      if (use_ms) {
        const T uk = u[k];
        ax += gx[p] * uk;
        ay += gy[p] * uk;
        az += gz[p] * uk;
      }
      if (use_ex) {
        const T c = kp[p];
        ax += c * m[3 * k];
        ay += c * m[3 * k + 1];
        az += c * m[3 * k + 2];
      }
    }
  }
  ax = group_sum(ax);
  ay = group_sum(ay);
  az = group_sum(az);
  if (!valid || lane != 0) return;
  const T Hx = ax + hx, Hy = ay + hy, Hz = az + hz;
  if (!(isfinite(Hx) && isfinite(Hy) && isfinite(Hz))) atomicOr(flag, FLAG_NONFINITE_OUT);
  if (MODE == 0) {
    H[3 * row] = Hx;
    H[3 * row + 1] = Hy;
    H[3 * row + 2] = Hz;
    return;
  }
  // dm/dt = -gam [m x H + alpha m x (m x H)]
  const T mx = m[3 * row], my = m[3 * row + 1], mz = m[3 * row + 2];
  const T cx = my * Hz - mz * Hy, cy = mz * Hx - mx * Hz, cz = mx * Hy - my * Hx;
  const T dx = my * cz - mz * cy, dy = mz * cx - mx * cz, dz = mx * cy - my * cx;
  const T kx = -gam * (cx + alpha * dx), ky = -gam * (cy + alpha * dy), kz = -gam * (cz + alpha * dz);
  const T sx = m0[3 * row], sy = m0[3 * row + 1], sz = m0[3 * row + 2];
  if (MODE == 1) {
    mnext[3 * row] = sx + cdt * kx;
    mnext[3 * row + 1] = sy + cdt * ky;
    mnext[3 * row + 2] = sz + cdt * kz;
    if (acc_init) {
      accb[3 * row] = bw * kx;
      accb[3 * row + 1] = bw * ky;
      accb[3 * row + 2] = bw * kz;
    } else {
      accb[3 * row] += bw * kx;
      accb[3 * row + 1] += bw * ky;
      accb[3 * row + 2] += bw * kz;
    }
  } else {
    const double nx = (double)sx + (double)dt6 * ((double)accb[3 * row] + (double)kx);
    const double ny = (double)sy + (double)dt6 * ((double)accb[3 * row + 1] + (double)ky);
    const double nz = (double)sz + (double)dt6 * ((double)accb[3 * row + 2] + (double)kz);
    const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
    m0[3 * row] = (T)(nx * inv);
    m0[3 * row + 1] = (T)(ny * inv);
    m0[3 * row + 2] = (T)(nz * inv);
  }
}

inline unsigned blocks_for(int64_t threads) { return (unsigned)((threads + kBlock - 1) / kBlock); }

}  // namespace

template <typename T>
void launch_charges(const DevOps<T>& d, const T* m, cudaStream_t st) {
  d.prof.begin(KID_CHARGES, st);
  k_charges<T><<<blocks_for(d.Np * kG), kBlock, 0, st>>>(d.Np, d.rowptr, d.col, d.wq[0], d.wq[1], d.wq[2], d.ea[0],
                                                         d.ea[1], d.ea[2], m, d.q, d.e, d.flag);
  d.prof.end(KID_CHARGES, st);
}

template <typename T>
void launch_anterp(const DevOps<T>& d, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np);
  d.prof.begin(KID_ANTERP, st);
#define PMFEM_ANTERP(PP)                                                                                \
  k_anterp<T, PP><<<nb, kBlock, 0, st>>>(d.Np, d.base, d.frac, d.q, d.grid, d.dims[0], d.dims[1], d.dims[2], \
                                         d.periodic[0], d.periodic[1], d.periodic[2])
  switch (d.p) {
    case 2: PMFEM_ANTERP(3); break;
    case 3: PMFEM_ANTERP(4); break;
    case 4: PMFEM_ANTERP(5); break;
    default: PMFEM_ANTERP(6); break;
  }
#undef PMFEM_ANTERP
  d.prof.end(KID_ANTERP, st);
}

template <typename T>
void launch_interp(const DevOps<T>& d, const T* m, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np * kG);
  d.prof.begin(KID_INTERP, st);
#define PMFEM_INTERP(PP)                                                                                          \
  k_interp<T, PP><<<nb, kBlock, 0, st>>>(d.Np, d.base, d.frac, d.grid, d.dims[0], d.dims[1], d.dims[2],          \
                                         d.periodic[0], d.periodic[1], d.periodic[2], d.rowptrC, d.colC, d.valC, \
                                         d.rowptrX, d.colX, d.valX, d.q, d.e, m, d.u)
  switch (d.p) {
    case 2: PMFEM_INTERP(3); break;
    case 3: PMFEM_INTERP(4); break;
    case 4: PMFEM_INTERP(5); break;
    default: PMFEM_INTERP(6); break;
  }
#undef PMFEM_INTERP
  d.prof.end(KID_INTERP, st);
}

template <typename T>
void launch_field(const DevOps<T>& d, const T* m, T* H, int comps, double hx, double hy, double hz, const RkArgs& rk,
                  cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np * kG);
  const int use_ms = (comps & 2) ? 1 : 0, use_ex = (comps & 1) ? 1 : 0;
  const T ax = (comps & 4) ? (T)hx : T(0), ay = (comps & 4) ? (T)hy : T(0), az = (comps & 4) ? (T)hz : T(0);
  T* m0 = (T*)rk.m0;
  T* mn = (T*)rk.mnext;
  T* acc = (T*)rk.acc;
  d.prof.begin(KID_FIELD, st);
  if (rk.mode == 0)
    k_field<T, 0><<<nb, kBlock, 0, st>>>(d.Np, d.rowptr, d.col, d.gr[0], d.gr[1], d.gr[2], d.kp, d.u, m, H, use_ms,
                                         use_ex, ax, ay, az, m0, mn, acc, (T)rk.cdt, (T)rk.bw, rk.acc_init,
                                         (T)rk.dt6, (T)rk.gam, (T)rk.alpha, d.flag);
  else if (rk.mode == 1)
    k_field<T, 1><<<nb, kBlock, 0, st>>>(d.Np, d.rowptr, d.col, d.gr[0], d.gr[1], d.gr[2], d.kp, d.u, m, H, use_ms,
                                         use_ex, ax, ay, az, m0, mn, acc, (T)rk.cdt, (T)rk.bw, rk.acc_init,
                                         (T)rk.dt6, (T)rk.gam, (T)rk.alpha, d.flag);
  else
    k_field<T, 2><<<nb, kBlock, 0, st>>>(d.Np, d.rowptr, d.col, d.gr[0], d.gr[1], d.gr[2], d.kp, d.u, m, H, use_ms,
                                         use_ex, ax, ay, az, m0, mn, acc, (T)rk.cdt, (T)rk.bw, rk.acc_init,
                                         (T)rk.dt6, (T)rk.gam, (T)rk.alpha, d.flag);
  d.prof.end(KID_FIELD, st);
}

#define PMFEM_INSTANTIATE(T)                                                                        \
  template void launch_charges<T>(const DevOps<T>&, const T*, cudaStream_t);                        \
  template void launch_anterp<T>(const DevOps<T>&, cudaStream_t);                                   \
  template void launch_interp<T>(const DevOps<T>&, const T*, cudaStream_t);                         \
  template void launch_field<T>(const DevOps<T>&, const T*, T*, int, double, double, double, const RkArgs&, \
                                cudaStream_t);
PMFEM_INSTANTIATE(double)
PMFEM_INSTANTIATE(float)
#undef PMFEM_INSTANTIATE

}  // namespace pmfem
