// Field-evaluation kernels for sm_103a: charges (Eq. 14a) with the touching-element part
// of Eq. 14c, projection onto the grid (BAIM step 1), interpolation plus precorrection
// (steps 3 and 4), and the gradient (Eq. 14d) + exchange (Eq. 8) pass with the fused
// RK4 stage update of the LLG equation (Eq. 2).  All arrays are in the internal
// box-sorted order except the C-ABI's m and H, which are permuted at the boundary.
#include <cmath>
#include <cstdio>

#include "device.hpp"

namespace pmfem {

namespace {

constexpr int kG = 8;          // lanes cooperating on one adjacency row
constexpr int kBlock = 256;
constexpr size_t kAnterpSmem = 96 * 1024;

template <typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, kG);
  return v;
}
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

// w[i] for a run-time i without indexing the register array dynamically
template <typename T, int P>
__device__ __forceinline__ T pick(const T (&w)[P], int i) {
  T r = w[0];
#pragma unroll
  for (int c = 1; c < P; ++c) r = (i == c) ? w[c] : r;
  return r;
}

__device__ __forceinline__ int wrap(int i, int N, bool per) {
  if (per) {
    if (i < 0) i += N;
    if (i >= N) i -= N;
  }
  return i;
}

__device__ __forceinline__ bool wrap_in(int& v, int N, bool per) {
  if (per) {
    if (v < 0) v += N;
    if (v >= N) v -= N;
    return true;
  }
  return v >= 0 && v < N;
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
template <typename T>
__global__ void __launch_bounds__(kBlock) k_charges(int64_t Np, const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const T* __restrict__ wx,
                                                   const T* __restrict__ wy, const T* __restrict__ wz,
                                                   const T* __restrict__ ex, const T* __restrict__ ey,
                                                   const T* __restrict__ ez, const V4<T>* __restrict__ m,
                                                   T* __restrict__ q, T* __restrict__ e) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kG;
  const int lane = threadIdx.x % kG;
  const bool valid = row < Np;
  T aq = 0, ae = 0;
  if (valid) {
    const int32_t b = rowptr[row], en = rowptr[row + 1];
    for (int32_t p = b + lane; p < en; p += kG) {
      const V4<T> mk = m[col[p]];
      aq += wx[p] * mk.x + wy[p] * mk.y + wz[p] * mk.z;
      ae += ex[p] * mk.x + ey[p] * mk.y + ez[p] * mk.z;
    }
  }
  aq = group_sum(aq);
  ae = group_sum(ae);
  if (valid && lane == 0) {
    q[row] = aq;
    e[row] = ae;
  }
}

// ---------------------------------------------------------------- projection (step 1)
// One block per tile of TY box rows x TZ box planes: its nodes are contiguous in the
// internal order; their stencils are accumulated in a shared-memory region covering the
// tile plus the stencil reach, then the region is added to the grid (periodic axes wrap).
template <typename T, int P>
__global__ void __launch_bounds__(kBlock) k_anterp_tiled(const int32_t* __restrict__ bstart,
                                                        const int32_t* __restrict__ base, const T* __restrict__ frac,
                                                        const T* __restrict__ q, T* __restrict__ grid, int N0, int N1,
                                                        int N2, bool p0, bool p1, bool p2, int TY, int TZ, int pl,
                                                        int pr) {
  extern __shared__ unsigned char smem_raw[];
  T* reg = reinterpret_cast<T*>(smem_raw);
  const int tile = blockIdx.x;
  const int NTY = N1 / TY;
  const int ty = tile % NTY, tz = tile / NTY;
  const int ox = -pl, oy = ty * TY - pl, oz = tz * TZ - pl;
  const int RX = N0 + pl + pr, RY = TY + pl + pr, RZ = TZ + pl + pr;
  const int R = RX * RY * RZ;
  for (int r = threadIdx.x; r < R; r += blockDim.x) reg[r] = T(0);
  __syncthreads();
  const int64_t boxes_per_tile = (int64_t)TY * TZ * N0;
  const int64_t n0 = bstart[tile * boxes_per_tile], n1 = bstart[(tile + 1) * boxes_per_tile];
  for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
    T w0[P], w1[P], w2[P];
    lagrange<T, P>(frac[3 * n], w0);
    lagrange<T, P>(frac[3 * n + 1], w1);
    lagrange<T, P>(frac[3 * n + 2], w2);
    const int b0 = base[3 * n], b1 = base[3 * n + 1], b2 = base[3 * n + 2];
    const T qn = q[n];
    const int lx = b0 - ox, ly = b1 - oy, lz = b2 - oz;
    if (lx >= 0 && lx + P <= RX && ly >= 0 && ly + P <= RY && lz >= 0 && lz + P <= RZ) {
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const T wz = w2[k] * qn;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          T* rowp = reg + lx + RX * ((ly + j) + RY * (lz + k));
          const T wzy = wz * w1[j];
#pragma unroll
          for (int i = 0; i < P; ++i) atomicAdd(rowp + i, wzy * w0[i]);
        }
      }
    } else {   // a stencil outside the tile region (rounding at a box edge): add directly
#pragma unroll
      for (int k = 0; k < P; ++k)
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
          for (int i = 0; i < P; ++i)
            atomicAdd(grid + wrap(b0 + i, N0, p0) +
                          (int64_t)N0 * (wrap(b1 + j, N1, p1) + (int64_t)N1 * wrap(b2 + k, N2, p2)),
                      w2[k] * qn * w1[j] * w0[i]);
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const T v = reg[r];
    if (v == T(0)) continue;
    const int rx = r % RX, ry = (r / RX) % RY, rz = r / (RX * RY);
    const int gx = wrap(ox + rx, N0, p0), gy = wrap(oy + ry, N1, p1), gz = wrap(oz + rz, N2, p2);
    if (gx < 0 || gx >= N0 || gy < 0 || gy >= N1 || gz < 0 || gz >= N2) continue;
    atomicAdd(grid + gx + (int64_t)N0 * (gy + (int64_t)N1 * gz), v);
  }
}

// fallback when a tile region does not fit in shared memory: direct global accumulation
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
// One warp per observer row.  Precorrection sources are the nodes of the (2 nb + 1)^2
// neighbouring box rows, each a contiguous node range [bstart(lo), bstart(hi + 1)); the
// row's values are stored in (dz, dy, x-segment, node) order, so a warp scan of the range
// lengths gives every lane the offset of its ranges.  The enumeration must match the
// host layout exactly (same loops, same wrap rules).
template <typename T, int P>
__global__ void __launch_bounds__(kBlock) k_interp(
    int64_t Np, const int32_t* __restrict__ box, const int32_t* __restrict__ base, const T* __restrict__ frac,
    const T* __restrict__ U, int N0, int N1, int N2, bool p0, bool p1, bool p2, int nb, int TY, int TZ,
    const int32_t* __restrict__ bstart, const int64_t* __restrict__ cptr, const T* __restrict__ cval,
    const int32_t* __restrict__ rowptrX, const int32_t* __restrict__ colX, const T* __restrict__ valX,
    const T* __restrict__ q, const T* __restrict__ e, const V4<T>* __restrict__ m, T* __restrict__ u, int* flag) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= Np) return;   // uniform per warp
  T acc = 0;
  // step 3: interpolation of the grid potential
  {
    T w0[P], w1[P], w2[P];
    lagrange<T, P>(frac[3 * row], w0);
    lagrange<T, P>(frac[3 * row + 1], w1);
    lagrange<T, P>(frac[3 * row + 2], w2);
    const int b0 = base[3 * row], b1 = base[3 * row + 1], b2 = base[3 * row + 2];
    for (int idx = lane; idx < P * P * P; idx += 32) {
      const int i = idx % P, j = (idx / P) % P, k = idx / (P * P);
      const int ix = wrap(b0 + i, N0, p0), iy = wrap(b1 + j, N1, p1), iz = wrap(b2 + k, N2, p2);
      acc += pick(w0, i) * pick(w1, j) * pick(w2, k) * U[ix + (int64_t)N0 * (iy + (int64_t)N1 * iz)];
    }
  }
  // step 4: point precorrection over the neighbouring box rows
  {
    const int bx = box[3 * row], by = box[3 * row + 1], bz = box[3 * row + 2];
    const int W = 2 * nb + 1, T2 = W * W;
    const int NTY = N1 / TY;
    int64_t off_base = cptr[row];
    const int64_t row_end = cptr[row + 1];
    for (int r0 = 0; r0 < T2; r0 += 32) {
      const int t = r0 + lane;
      int a0 = 0, a1 = 0, c0 = 0, c1 = 0;   // node ranges [a0, a1) and [c0, c1)
      int len = 0;
      if (t < T2) {
        int z = bz + t / W - nb, y = by + t % W - nb;
        if (wrap_in(z, N2, p2) && wrap_in(y, N1, p1)) {
          const int64_t rowbox = ((((int64_t)(z / TZ) * NTY + y / TY) * TZ + z % TZ) * TY + y % TY) * N0;
          int lo = bx - nb, hi = bx + nb;
          int lo2 = 0, hi2 = -1;               // second x-segment after a periodic wrap
          if (!p0) {
            lo = lo < 0 ? 0 : lo;
            hi = hi > N0 - 1 ? N0 - 1 : hi;
          } else if (lo < 0) {
            lo2 = 0, hi2 = hi, lo = lo + N0, hi = N0 - 1;
          } else if (hi >= N0) {
            lo2 = 0, hi2 = hi - N0, hi = N0 - 1;
          }
          if (lo <= hi) {
            a0 = bstart[rowbox + lo];
            a1 = bstart[rowbox + hi + 1];
          }
          if (lo2 <= hi2) {
            c0 = bstart[rowbox + lo2];
            c1 = bstart[rowbox + hi2 + 1];
          }
          len = (a1 - a0) + (c1 - c0);
        }
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      int64_t off = off_base + (incl - len);
      if (off + len > row_end) {   // enumeration disagrees with the stored layout
        atomicOr(flag, FLAG_LAYOUT);
        a1 = a0;
        c1 = c0;
      }
      for (int k = a0; k < a1; ++k, ++off) acc += cval[off] * q[k];
      for (int k = c0; k < c1; ++k, ++off) acc += cval[off] * q[k];
      off_base += total;
    }
  }
  // near-element entries beyond the adjacency pattern
  for (int32_t p = rowptrX[row] + lane; p < rowptrX[row + 1]; p += 32) {
    const V4<T> mk = m[colX[p]];
    acc += valX[3 * p] * mk.x + valX[3 * p + 1] * mk.y + valX[3 * p + 2] * mk.z;
  }
  acc = warp_sum(acc);
  if (lane == 0) u[row] = acc + e[row];
}

// ---------------------------------------------------------------- gradient + exchange + RK4
// Both operators annihilate constants (rows of the gradient and of the Laplacian sum to
// zero), so they act on differences to the row's own value: the same result in exact
// arithmetic, without the cancellation of large terms in floating point.
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock) k_field(int64_t Np, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ col, const T* __restrict__ gx,
                                                 const T* __restrict__ gy, const T* __restrict__ gz,
                                                 const T* __restrict__ kp, const T* __restrict__ u,
                                                 const V4<T>* __restrict__ m, const int32_t* __restrict__ perm,
                                                 T* __restrict__ H, int use_ms, int use_ex, T hx, T hy, T hz,
                                                 V4<T>* __restrict__ m0, V4<T>* __restrict__ mnext,
                                                 V4<T>* __restrict__ accb, T cdt, T bw, int acc_init, T dt6, T gam,
                                                 T alpha, int* flag) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kG;
  const int lane = threadIdx.x % kG;
  const bool valid = row < Np;
  T ax = 0, ay = 0, az = 0;
  V4<T> mn = {0, 0, 0, 0};
  if (valid) {
    const int32_t b = rowptr[row], en = rowptr[row + 1];
    const T un = use_ms ? u[row] : T(0);
    mn = m[row];
    for (int32_t p = b + lane; p < en; p += kG) {
      const int32_t k = col[p];
      if (use_ms) {
        const T du = u[k] - un;
        ax += gx[p] * du;
        ay += gy[p] * du;
        az += gz[p] * du;
      }
      if (use_ex) {
        const T c = kp[p];
        const V4<T> mk = m[k];
        ax += c * (mk.x - mn.x);
        ay += c * (mk.y - mn.y);
        az += c * (mk.z - mn.z);
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
    const int64_t o = 3 * (int64_t)perm[row];
    H[o] = Hx;
    H[o + 1] = Hy;
    H[o + 2] = Hz;
    return;
  }
  // dm/dt = -gam [m x H + alpha m x (m x H)]
  const T cx = mn.y * Hz - mn.z * Hy, cy = mn.z * Hx - mn.x * Hz, cz = mn.x * Hy - mn.y * Hx;
  const T dx = mn.y * cz - mn.z * cy, dy = mn.z * cx - mn.x * cz, dz = mn.x * cy - mn.y * cx;
  const T kx = -gam * (cx + alpha * dx), ky = -gam * (cy + alpha * dy), kz = -gam * (cz + alpha * dz);
  const V4<T> s = m0[row];
  if (MODE == 1) {
    mnext[row] = V4<T>{s.x + cdt * kx, s.y + cdt * ky, s.z + cdt * kz, T(0)};
    if (acc_init) {
      accb[row] = V4<T>{bw * kx, bw * ky, bw * kz, T(0)};
    } else {
      const V4<T> a = accb[row];
      accb[row] = V4<T>{a.x + bw * kx, a.y + bw * ky, a.z + bw * kz, T(0)};
    }
  } else {
    const V4<T> a = accb[row];
    const double nx = (double)s.x + (double)dt6 * ((double)a.x + (double)kx);
    const double ny = (double)s.y + (double)dt6 * ((double)a.y + (double)ky);
    const double nz = (double)s.z + (double)dt6 * ((double)a.z + (double)kz);
    const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
    m0[row] = V4<T>{(T)(nx * inv), (T)(ny * inv), (T)(nz * inv), T(0)};
  }
}

inline unsigned blocks_for(int64_t threads) { return (unsigned)((threads + kBlock - 1) / kBlock); }

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t anterp_smem_budget() { return kAnterpSmem; }

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
  d.prof.begin(KID_CHARGES, st);
  k_charges<T><<<blocks_for(d.Np * kG), kBlock, 0, st>>>(d.Np, d.rowptr, d.col, d.wq[0], d.wq[1], d.wq[2], d.ea[0],
                                                         d.ea[1], d.ea[2], m, d.q, d.e);
  d.prof.end(KID_CHARGES, st);
}

template <typename T>
void launch_anterp(const DevOps<T>& d, cudaStream_t st) {
  d.prof.begin(KID_ANTERP, st);
  const int N0 = d.dims[0], N1 = d.dims[1], N2 = d.dims[2];
  if (d.tiled) {
    const int RX = N0 + d.pl + d.pr, RY = d.TY + d.pl + d.pr, RZ = d.TZ + d.pl + d.pr;
    const size_t sm = (size_t)RX * RY * RZ * sizeof(T);
    const unsigned ntiles = (unsigned)((N1 / d.TY) * (N2 / d.TZ));
#define PMFEM_ANTERP_T(PP)                                                                                     \
  set_smem(k_anterp_tiled<T, PP>, sm);                                                                         \
  k_anterp_tiled<T, PP><<<ntiles, kBlock, sm, st>>>(d.bstart, d.base, d.frac, d.q, d.grid, N0, N1, N2,          \
                                                    d.periodic[0], d.periodic[1], d.periodic[2], d.TY, d.TZ, d.pl, \
                                                    d.pr)
    switch (d.p) {
      case 2: PMFEM_ANTERP_T(3); break;
      case 3: PMFEM_ANTERP_T(4); break;
      case 4: PMFEM_ANTERP_T(5); break;
      default: PMFEM_ANTERP_T(6); break;
    }
#undef PMFEM_ANTERP_T
  } else {
    const unsigned nb = blocks_for(d.Np);
#define PMFEM_ANTERP(PP)                                                                                    \
  k_anterp<T, PP><<<nb, kBlock, 0, st>>>(d.Np, d.base, d.frac, d.q, d.grid, N0, N1, N2, d.periodic[0],     \
                                         d.periodic[1], d.periodic[2])
    switch (d.p) {
      case 2: PMFEM_ANTERP(3); break;
      case 3: PMFEM_ANTERP(4); break;
      case 4: PMFEM_ANTERP(5); break;
      default: PMFEM_ANTERP(6); break;
    }
#undef PMFEM_ANTERP
  }
  d.prof.end(KID_ANTERP, st);
}

template <typename T>
void launch_interp(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np * 32);
  d.prof.begin(KID_INTERP, st);
#define PMFEM_INTERP(PP)                                                                                     \
  k_interp<T, PP><<<nb, kBlock, 0, st>>>(d.Np, d.box, d.base, d.frac, d.grid, d.dims[0], d.dims[1], d.dims[2], \
                                         d.periodic[0], d.periodic[1], d.periodic[2], d.nb, d.TY, d.TZ,          \
                                         d.bstart, d.cptr, d.cval, d.rowptrX, d.colX, d.valX, d.q, d.e, m, d.u, d.flag)
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
void launch_field(const DevOps<T>& d, const V4<T>* m, T* H, int comps, double hx, double hy, double hz,
                  const RkArgs& rk, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np * kG);
  const int use_ms = (comps & 2) ? 1 : 0, use_ex = (comps & 1) ? 1 : 0;
  const T ax = (comps & 4) ? (T)hx : T(0), ay = (comps & 4) ? (T)hy : T(0), az = (comps & 4) ? (T)hz : T(0);
  V4<T>* m0 = (V4<T>*)rk.m0;
  V4<T>* mn = (V4<T>*)rk.mnext;
  V4<T>* acc = (V4<T>*)rk.acc;
  d.prof.begin(KID_FIELD, st);
#define PMFEM_FIELD(MODE)                                                                                       \
  k_field<T, MODE><<<nb, kBlock, 0, st>>>(d.Np, d.rowptr, d.col, d.gr[0], d.gr[1], d.gr[2], d.kp, d.u, m, d.perm, \
                                          H, use_ms, use_ex, ax, ay, az, m0, mn, acc, (T)rk.cdt, (T)rk.bw,         \
                                          rk.acc_init, (T)rk.dt6, (T)rk.gam, (T)rk.alpha, d.flag)
  if (rk.mode == 0) PMFEM_FIELD(0);
  else if (rk.mode == 1) PMFEM_FIELD(1);
  else PMFEM_FIELD(2);
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
