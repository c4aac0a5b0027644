// Field-evaluation kernels for sm_103a: charges (Eq. 14a) with the touching-element part
// of Eq. 14c, projection onto the grid (BAIM step 1), interpolation plus precorrection
// (steps 3 and 4), and the gradient (Eq. 14d) + exchange (Eq. 8) pass with the fused
// RK4 stage update of the LLG equation (Eq. 2).
//
// Layout: unknowns in the internal box-sorted order (the C-ABI's m and H are permuted
// at the boundary); sparse rows in SELL-32, one thread per row, so that at every step j
// the 32 threads of a warp read 32 consecutive values (one 128-byte segment in FP32) and
// each thread has many independent loads in flight.  The projection is a gather: each
// grid point sums over the nodes whose stencil covers it, so there are no atomics (except
// for a short exception list) and the field is bitwise reproducible.
#include <cmath>
#include <cstdio>

#include "device.hpp"

namespace pmfem {

namespace {

constexpr int kBlock = 256;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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



// sum_j val[o_j] * x[b + delta[o_j]] over one SELL row, o_j = o + 32 j: the value and
// column loads of a batch of B elements are issued together, then their B gathers, so
// each thread keeps 2B independent loads in flight instead of one dependent pair
template <int B, typename T, typename CT>
__device__ __forceinline__ T sell_dot(const T* __restrict__ val, const CT* __restrict__ dcol,
                                      const T* __restrict__ x, int64_t b, int64_t o, int n) {
  T acc = 0;
  int j = 0;
  for (; j + B <= n; j += B, o += 32 * B) {
    T v[B];
    int64_t c[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      v[k] = __ldcs(val + o + 32 * k);
      c[k] = b + (int64_t)__ldcs(dcol + o + 32 * k);
    }
#pragma unroll
    for (int k = 0; k < B; ++k) acc += v[k] * __ldg(x + c[k]);
  }
  for (; j < n; ++j, o += 32) acc += __ldcs(val + o) * __ldg(x + b + __ldcs(dcol + o));
  return acc;
}

// ---------------------------------------------------------------- boundary permutations
template <typename T>
__global__ void __launch_bounds__(kBlock) k_perm_in(int64_t Np, const int32_t* __restrict__ perm,
                                                   const T* __restrict__ mu, V4<T>* __restrict__ m, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int64_t u = perm[i];
  V4<T> v;
  v.x = mu[3 * u];
  v.y = mu[3 * u + 1];
  v.z = mu[3 * u + 2];
  v.w = T(0);
  if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) atomicOr(flag, FLAG_NONFINITE_IN);
  m[i] = v;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_perm_out(int64_t Np, const int32_t* __restrict__ perm,
                                                    const V4<T>* __restrict__ m, T* __restrict__ mu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int64_t u = perm[i];
  const V4<T> v = m[i];
  mu[3 * u] = v.x;
  mu[3 * u + 1] = v.y;
  mu[3 * u + 2] = v.z;
}

// ---------------------------------------------------------------- charges
// q = W^q M (Eq. 14a) and e = E M (touching-element part of Eq. 14c) on the adjacency.
template <typename T, typename CT>
__global__ void __launch_bounds__(kBlock) k_charges(int64_t Np, const int32_t* __restrict__ len,
                                                   const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                                   const T* __restrict__ wx, const T* __restrict__ wy,
                                                   const T* __restrict__ wz, const T* __restrict__ ex,
                                                   const T* __restrict__ ey, const T* __restrict__ ez,
                                                   const V4<T>* __restrict__ m, T* __restrict__ q, T* __restrict__ e) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int n = len[i];
  int64_t o = off[i >> 5] + (i & 31);
  T aq = 0, ae = 0;
#pragma unroll 4
  for (int j = 0; j < n; ++j, o += 32) {
    const V4<T> mk = m[i + (int64_t)__ldcs(dcol + o)];
    aq += __ldcs(wx + o) * mk.x + __ldcs(wy + o) * mk.y + __ldcs(wz + o) * mk.z;
    ae += __ldcs(ex + o) * mk.x + __ldcs(ey + o) * mk.y + __ldcs(ez + o) * mk.z;
  }
  q[i] = aq;
  e[i] = ae;
}

// ---------------------------------------------------------------- projection (step 1)
// Q = P^T q as a gather: grid point g (one thread, SELL-32 over grid points) sums w q over
// the nodes whose stencil covers it (the nodes of the boxes [g - pr, g + pl] per axis,
// enumerated at set-up).  No atomics: every grid value has one writer.
template <typename T, typename CT>
__global__ void __launch_bounds__(kBlock) k_project(int64_t G, const int32_t* __restrict__ map,
                                                   const int32_t* __restrict__ len, const int32_t* __restrict__ base,
                                                   const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                                   const T* __restrict__ pw, const T* __restrict__ q,
                                                   T* __restrict__ grid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G) return;
  const int64_t g = map ? (int64_t)map[t] : t;   // grid point of this thread (null map: identity)
  const int n = len[t];
  T acc = 0;
  if (n > 0) acc = sell_dot<8>(pw, dcol, q, (int64_t)base[t], off[t >> 5] + (t & 31), n);
  grid[g] = acc;
}

// nodes whose stencil is not aligned with their box (rare rounding cases)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_project_exc(int64_t n, const int32_t* __restrict__ node,
                                                       const int64_t* __restrict__ gidx, const T* __restrict__ w,
                                                       const T* __restrict__ q, T* __restrict__ grid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  atomicAdd(grid + gidx[t], w[t] * q[node[t]]);
}

// ---------------------------------------------------------------- interpolation + precorrection
// One thread per observer row (thread t handles row map[t], or row t when the operator
// keeps the box order): the (p+1)^3 stencil gathers from the grid potential, then the row
// of the point precorrection.
template <typename T, int P, typename CT>
__global__ void __launch_bounds__(kBlock) k_interp(
    int64_t Np, const int32_t* __restrict__ map, const int32_t* __restrict__ base, const T* __restrict__ frac,
    const T* __restrict__ U, int N0, int N1, int N2, bool p0, bool p1, bool p2, const int32_t* __restrict__ clen,
    const int64_t* __restrict__ coff, const CT* __restrict__ dcol, const T* __restrict__ cval,
    const int32_t* __restrict__ rowptrX, const int32_t* __restrict__ colX, const T* __restrict__ valX,
    const T* __restrict__ q, const T* __restrict__ e, const V4<T>* __restrict__ m, T* __restrict__ u) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Np) return;
  const int64_t i = map ? (int64_t)map[t] : t;   // a null map is the identity
  T acc = 0;
  {  // step 3: interpolation of the grid potential
    T w0[P], w1[P], w2[P];
    lagrange<T, P>(frac[3 * i], w0);
    lagrange<T, P>(frac[3 * i + 1], w1);
    lagrange<T, P>(frac[3 * i + 2], w2);
    const int b0 = base[3 * i], b1 = base[3 * i + 1], b2 = base[3 * i + 2];
    int ix[P];
#pragma unroll
    for (int a = 0; a < P; ++a) ix[a] = wrap(b0 + a, N0, p0);
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int64_t zo = (int64_t)N1 * wrap(b2 + c, N2, p2);
#pragma unroll
      for (int b = 0; b < P; ++b) {
        const T* rowp = U + (int64_t)N0 * (wrap(b1 + b, N1, p1) + zo);
        T s = 0;
#pragma unroll
        for (int a = 0; a < P; ++a) s += w0[a] * __ldg(rowp + ix[a]);
        acc += w2[c] * w1[b] * s;
      }
    }
  }
  {  // step 4: point precorrection (SELL-32 row)
    acc += sell_dot<8>(cval, dcol, q, i, coff[t >> 5] + (t & 31), clen[t]);
  }
  // near-element entries beyond the adjacency pattern
  for (int32_t p = rowptrX[i]; p < rowptrX[i + 1]; ++p) {
    const V4<T> mk = m[colX[p]];
    acc += valX[3 * p] * mk.x + valX[3 * p + 1] * mk.y + valX[3 * p + 2] * mk.z;
  }
  u[i] = acc + e[i];
}

// ---------------------------------------------------------------- gradient + exchange + RK4
// Both operators annihilate constants (rows of the gradient and of the Laplacian sum to
// zero), so they act on differences to the row's own value: the same result in exact
// arithmetic, without the cancellation of large terms in floating point.
template <typename T, int MODE, typename CT>
__global__ void __launch_bounds__(kBlock) k_field(int64_t Np, const int32_t* __restrict__ len,
                                                 const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                                 const T* __restrict__ gx, const T* __restrict__ gy,
                                                 const T* __restrict__ gz, const T* __restrict__ kp,
                                                 const T* __restrict__ u, const V4<T>* __restrict__ m,
                                                 const int32_t* __restrict__ perm, T* __restrict__ H, int use_ms,
                                                 int use_ex, T hx, T hy, T hz, V4<T>* __restrict__ m0,
                                                 V4<T>* __restrict__ mnext, V4<T>* __restrict__ accb, T cdt, T bw,
                                                 int acc_init, T dt6, T gam, T alpha, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int n = len[i];
  int64_t o = off[i >> 5] + (i & 31);
  const V4<T> mn = m[i];
  const T un = use_ms ? u[i] : T(0);
  T ax = 0, ay = 0, az = 0;
  if (use_ms && use_ex) {
#pragma unroll 4
    for (int j = 0; j < n; ++j, o += 32) {
      const int64_t k = i + (int64_t)__ldcs(dcol + o);
      const T du = __ldg(u + k) - un;
      const V4<T> mk = m[k];
      const T c = __ldcs(kp + o);
      ax += __ldcs(gx + o) * du + c * (mk.x - mn.x);
      ay += __ldcs(gy + o) * du + c * (mk.y - mn.y);
      az += __ldcs(gz + o) * du + c * (mk.z - mn.z);
    }
  } else if (use_ms) {
#pragma unroll 4
    for (int j = 0; j < n; ++j, o += 32) {
      const T du = __ldg(u + i + __ldcs(dcol + o)) - un;
      ax += __ldcs(gx + o) * du;
      ay += __ldcs(gy + o) * du;
      az += __ldcs(gz + o) * du;
    }
  } else if (use_ex) {
#pragma unroll 4
    for (int j = 0; j < n; ++j, o += 32) {
      const V4<T> mk = m[i + (int64_t)__ldcs(dcol + o)];
      const T c = __ldcs(kp + o);
      ax += c * (mk.x - mn.x);
      ay += c * (mk.y - mn.y);
      az += c * (mk.z - mn.z);
    }
  }
  const T Hx = ax + hx, Hy = ay + hy, Hz = az + hz;
  if (!(isfinite(Hx) && isfinite(Hy) && isfinite(Hz))) atomicOr(flag, FLAG_NONFINITE_OUT);
  if (MODE == 0) {
    const int64_t uo = 3 * (int64_t)perm[i];
    H[uo] = Hx;
    H[uo + 1] = Hy;
    H[uo + 2] = Hz;
    return;
  }
  // dm/dt = -gam [m x H + alpha m x (m x H)]
  const T cx = mn.y * Hz - mn.z * Hy, cy = mn.z * Hx - mn.x * Hz, cz = mn.x * Hy - mn.y * Hx;
  const T dx = mn.y * cz - mn.z * cy, dy = mn.z * cx - mn.x * cz, dz = mn.x * cy - mn.y * cx;
  const T kx = -gam * (cx + alpha * dx), ky = -gam * (cy + alpha * dy), kz = -gam * (cz + alpha * dz);
  const V4<T> s = m0[i];
  if (MODE == 1) {
    mnext[i] = V4<T>{s.x + cdt * kx, s.y + cdt * ky, s.z + cdt * kz, T(0)};
    if (acc_init) {
      accb[i] = V4<T>{bw * kx, bw * ky, bw * kz, T(0)};
    } else {
      const V4<T> a = accb[i];
      accb[i] = V4<T>{a.x + bw * kx, a.y + bw * ky, a.z + bw * kz, T(0)};
    }
  } else {
    const V4<T> a = accb[i];
    const double nx = (double)s.x + (double)dt6 * ((double)a.x + (double)kx);
    const double ny = (double)s.y + (double)dt6 * ((double)a.y + (double)ky);
    const double nz = (double)s.z + (double)dt6 * ((double)a.z + (double)kz);
    const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
    m0[i] = V4<T>{(T)(nx * inv), (T)(ny * inv), (T)(nz * inv), T(0)};
  }
}

inline unsigned blocks_for(int64_t threads) { return (unsigned)((threads + kBlock - 1) / kBlock); }

}  // namespace

template <typename T>
void launch_perm_in(const DevOps<T>& d, const T* m_user, V4<T>* m, cudaStream_t st) {
  d.prof.begin(KID_PERM, st);
  k_perm_in<T><<<blocks_for(d.Np), kBlock, 0, st>>>(d.Np, d.perm, m_user, m, d.flag);
  d.prof.end(KID_PERM, st);
}

template <typename T>
void launch_perm_out(const DevOps<T>& d, const V4<T>* m, T* m_user, cudaStream_t st) {
  d.prof.begin(KID_PERM, st);
  k_perm_out<T><<<blocks_for(d.Np), kBlock, 0, st>>>(d.Np, d.perm, m, m_user);
  d.prof.end(KID_PERM, st);
}

template <typename T>
void launch_charges(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const DevSell<T>& A = d.adj;
  d.prof.begin(KID_CHARGES, st);
  if (A.col16)
    k_charges<T, int16_t><<<blocks_for(d.Np), kBlock, 0, st>>>(d.Np, A.len, A.off, (const int16_t*)A.delta, A.val[0],
                                                               A.val[1], A.val[2], A.val[3], A.val[4], A.val[5], m,
                                                               d.q, d.e);
  else
    k_charges<T, int32_t><<<blocks_for(d.Np), kBlock, 0, st>>>(d.Np, A.len, A.off, (const int32_t*)A.delta, A.val[0],
                                                               A.val[1], A.val[2], A.val[3], A.val[4], A.val[5], m,
                                                               d.q, d.e);
  d.prof.end(KID_CHARGES, st);
}

template <typename T>
void launch_anterp(const DevOps<T>& d, cudaStream_t st) {
  const DevSell<T>& Pm = d.pro;
  d.prof.begin(KID_ANTERP, st);
  const int64_t G = Pm.rows;
  if (Pm.col16)
    k_project<T, int16_t><<<blocks_for(G), kBlock, 0, st>>>(G, Pm.map, Pm.len, Pm.base, Pm.off,
                                                            (const int16_t*)Pm.delta, Pm.val[0], d.q, d.grid);
  else
    k_project<T, int32_t><<<blocks_for(G), kBlock, 0, st>>>(G, Pm.map, Pm.len, Pm.base, Pm.off,
                                                            (const int32_t*)Pm.delta, Pm.val[0], d.q, d.grid);
  if (d.nx_exc > 0)
    k_project_exc<T><<<blocks_for(d.nx_exc), kBlock, 0, st>>>(d.nx_exc, d.xnode, d.xgrid, d.xw, d.q, d.grid);
  d.prof.end(KID_ANTERP, st);
}

template <typename T>
void launch_interp(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const DevSell<T>& C = d.cor;
  const unsigned nb = blocks_for(d.Np);
  d.prof.begin(KID_INTERP, st);
#define PMFEM_INTERP(PP, CT)                                                                                      \
  k_interp<T, PP, CT><<<nb, kBlock, 0, st>>>(d.Np, C.map, d.base, d.frac, d.grid, d.dims[0], d.dims[1], d.dims[2], \
                                             d.periodic[0], d.periodic[1], d.periodic[2], C.len, C.off,           \
                                             (const CT*)C.delta, C.val[0], d.rowptrX, d.colX, d.valX, d.q, d.e, m, \
                                             d.u)
#define PMFEM_INTERP_P(CT)              \
  switch (d.p) {                        \
    case 2: PMFEM_INTERP(3, CT); break; \
    case 3: PMFEM_INTERP(4, CT); break; \
    case 4: PMFEM_INTERP(5, CT); break; \
    default: PMFEM_INTERP(6, CT); break; \
  }
  if (C.col16) {
    PMFEM_INTERP_P(int16_t)
  } else {
    PMFEM_INTERP_P(int32_t)
  }
#undef PMFEM_INTERP_P
#undef PMFEM_INTERP
  d.prof.end(KID_INTERP, st);
}

template <typename T>
void launch_field(const DevOps<T>& d, const V4<T>* m, T* H, int comps, double hx, double hy, double hz,
                  const RkArgs& rk, cudaStream_t st) {
  const DevSell<T>& A = d.adj;
  const unsigned nb = blocks_for(d.Np);
  const int use_ms = (comps & 2) ? 1 : 0, use_ex = (comps & 1) ? 1 : 0;
  const T ax = (comps & 4) ? (T)hx : T(0), ay = (comps & 4) ? (T)hy : T(0), az = (comps & 4) ? (T)hz : T(0);
  V4<T>* m0 = (V4<T>*)rk.m0;
  V4<T>* mn = (V4<T>*)rk.mnext;
  V4<T>* acc = (V4<T>*)rk.acc;
  d.prof.begin(KID_FIELD, st);
#define PMFEM_FIELD(MODE, CT)                                                                                     \
  k_field<T, MODE, CT><<<nb, kBlock, 0, st>>>(d.Np, A.len, A.off, (const CT*)A.delta, A.val[6], A.val[7], A.val[8], \
                                              A.val[9], d.u, m, d.perm, H, use_ms, use_ex, ax, ay, az, m0, mn, acc, \
                                              (T)rk.cdt, (T)rk.bw, rk.acc_init, (T)rk.dt6, (T)rk.gam, (T)rk.alpha,   \
                                              d.flag)
#define PMFEM_FIELD_M(CT)                           \
  if (rk.mode == 0) PMFEM_FIELD(0, CT);             \
  else if (rk.mode == 1) PMFEM_FIELD(1, CT);        \
  else PMFEM_FIELD(2, CT);
  if (A.col16) {
    PMFEM_FIELD_M(int16_t)
  } else {
    PMFEM_FIELD_M(int32_t)
  }
#undef PMFEM_FIELD_M
#undef PMFEM_FIELD
  d.prof.end(KID_FIELD, st);
}

#define PMFEM_INSTANTIATE(T)                                                                          \
  template void launch_perm_in<T>(const DevOps<T>&, const T*, V4<T>*, cudaStream_t);                 \
  template void launch_perm_out<T>(const DevOps<T>&, const V4<T>*, T*, cudaStream_t);                \
  template void launch_charges<T>(const DevOps<T>&, const V4<T>*, cudaStream_t);                     \
  template void launch_anterp<T>(const DevOps<T>&, cudaStream_t);                                    \
  template void launch_interp<T>(const DevOps<T>&, const V4<T>*, cudaStream_t);                      \
  template void launch_field<T>(const DevOps<T>&, const V4<T>*, T*, int, double, double, double, const RkArgs&, \
                                cudaStream_t);
PMFEM_INSTANTIATE(double)
PMFEM_INSTANTIATE(float)
#undef PMFEM_INSTANTIATE

}  // namespace pmfem
