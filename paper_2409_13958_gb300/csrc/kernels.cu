// Field-evaluation kernels for sm_103a: charges (Eq. 14a) with the touching-element part
// of Eq. 14c, projection onto the grid (BAIM step 1), interpolation plus precorrection
// (steps 3 and 4: one fused kernel, or a precorrection pass that can run beside the
// projection and FFT followed by a stencil pass), and the gradient (Eq. 14d) + exchange
// (Eq. 8) pass with the fused RK4 stage update of the LLG equation (Eq. 2).
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
#include "sell.cuh"

namespace pmfem {

namespace {

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
// the charges kernel asks for 4 resident blocks per SM (64 registers; measured 82 -> 77 us
// on the 1M-node wire against the compiler's own 66 registers and 3 blocks)
#ifndef PMFEM_CHARGES_MINB
#define PMFEM_CHARGES_MINB 4
#endif
#define PMFEM_CHARGES_LB __launch_bounds__(kBlock, PMFEM_CHARGES_MINB)
template <typename T, typename CT, typename VT>
__global__ void PMFEM_CHARGES_LB k_charges(int64_t Np, const int32_t* __restrict__ len,
                                                   const int32_t* __restrict__ base,
                                                   const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                                   const VT* __restrict__ wx, const VT* __restrict__ wy,
                                                   const VT* __restrict__ wz, const VT* __restrict__ ex,
                                                   const VT* __restrict__ ey, const VT* __restrict__ ez,
                                                   const V4<T>* __restrict__ m, T* __restrict__ q, T* __restrict__ e) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  charges_row<T, CT, VT>(i, 0, (int32_t)Np, len, base, off, dcol, wx, wy, wz, ex, ey, ez, m, q, e);
}

// ---------------------------------------------------------------- projection (step 1)
// One thread per grid point (SELL-32 over grid points; thread t handles point map[t], or
// t when the operator keeps the grid order).  No atomics: every grid value has one writer.
template <typename T, typename CT, typename VT>
__global__ void __launch_bounds__(kBlock) k_project(int64_t G, int64_t Np, const int32_t* __restrict__ map,
                                                   const int32_t* __restrict__ len, const int32_t* __restrict__ base,
                                                   const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                                   const VT* __restrict__ pw, const T* __restrict__ q,
                                                   T* __restrict__ grid) {
  pdl_enter();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G) return;
  const int64_t g = map ? (int64_t)map[t] : t;
  project_row<T, CT, VT>(t, g, 0, (int32_t)Np, len, base, off, dcol, pw, q, grid);
}

// nodes whose stencil is not aligned with their box (rare rounding cases)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_project_exc(int64_t n, const int32_t* __restrict__ node,
                                                       const int64_t* __restrict__ gidx, const T* __restrict__ w,
                                                       const T* __restrict__ q, T* __restrict__ grid) {
  pdl_enter();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  atomicAdd(grid + gidx[t], w[t] * q[node[t]]);
}

// ---------------------------------------------------------------- interpolation + precorrection
// Fused form: one thread per precorrection row t (node map[t]) does both steps, so u is
// written once and the node data are read once.  The FP32 kernel with stencils of up to 4
// points per axis asks for PMFEM_INTERP_MINB resident blocks per SM (a register cap).
#ifndef PMFEM_INTERP_MINB
#define PMFEM_INTERP_MINB 5
#endif
// Stages of the shared-memory pipeline of the precorrection streams, by stored value type
// (0: register loads).  Measured on the 1M-node wire: bfloat16 values gain 10% with three
// stages, FP64 2% with two; FP32 values lose 12-17% (the buffer takes L1 that the gathers of
// q hit), so they keep the register loads.
#ifndef PMFEM_COR_PIPE_F32
#define PMFEM_COR_PIPE_F32 0
#endif
#ifndef PMFEM_COR_PIPE_F64
#define PMFEM_COR_PIPE_F64 2
#endif
#ifndef PMFEM_COR_PIPE_BF16
#define PMFEM_COR_PIPE_BF16 3
#endif
template <typename VT>
__host__ __device__ constexpr int cor_pipe() {
  return sizeof(VT) == 2 ? PMFEM_COR_PIPE_BF16 : sizeof(VT) == 8 ? PMFEM_COR_PIPE_F64 : PMFEM_COR_PIPE_F32;
}
#define PMFEM_INTERP_PARAMS                                                                                      \
  int64_t Np, const int32_t *__restrict__ map, const int32_t *__restrict__ base, const T *__restrict__ frac,      \
      const T *__restrict__ U, int N0, int N1, int N2, bool p0, bool p1, bool p2,                                \
      const int32_t *__restrict__ clen, const int32_t *__restrict__ cbase, const int64_t *__restrict__ coff,     \
      const CT *__restrict__ dcol, const VT *__restrict__ cval, const int32_t *__restrict__ rowptrX,             \
      const int32_t *__restrict__ colX, const T *__restrict__ valX, const T *__restrict__ q,                      \
      const T *__restrict__ e, const V4<T> *m, T *uw
#define PMFEM_INTERP_BODY                                                                                         \
  extern __shared__ __align__(16) unsigned char pipe_raw[];                                                      \
  pdl_enter();                                                                                                    \
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;                                              \
  if (t >= Np) return;                                                                                            \
  const int64_t i = map ? (int64_t)map[t] : t;                                                                    \
  interp_row<T, P, CT, VT, cor_pipe<VT>()>(                                                                      \
      t, i, 0, (int32_t)Np, base, frac, U, N0, N1, N2, p0, p1, p2, clen, cbase, coff, dcol, cval, rowptrX, colX,  \
      valX, q, e, m, uw, pipe_raw + (threadIdx.x >> 5) * (cor_pipe<VT>() * PipeStage<VT, CT>::BYTES));
template <typename T, int P, typename CT, typename VT>
__global__ void __launch_bounds__(kBlock, PMFEM_INTERP_MINB) k_interp_capped(PMFEM_INTERP_PARAMS) {
  PMFEM_INTERP_BODY
}
template <typename T, int P, typename CT, typename VT>
__global__ void __launch_bounds__(kBlock) k_interp(PMFEM_INTERP_PARAMS) {
  PMFEM_INTERP_BODY
}
#undef PMFEM_INTERP_BODY
#undef PMFEM_INTERP_PARAMS
template <typename T, int P, typename CT, typename VT>
constexpr auto interp_kernel() {
  if constexpr (sizeof(T) == 4 && P <= 4)
    return k_interp_capped<T, P, CT, VT>;
  else
    return k_interp<T, P, CT, VT>;
}

// ---------------------------------------------------------------- the two-pass form
// Precorrection pass (one thread per precorrection row, as in the fused kernel, without the
// stencil) and stencil pass (one thread per node in the internal order).
#define PMFEM_PRECORR_PARAMS                                                                                    \
  int64_t Np, const int32_t *__restrict__ map, const int32_t *__restrict__ clen,                               \
      const int32_t *__restrict__ cbase, const int64_t *__restrict__ coff, const CT *__restrict__ dcol,           \
      const VT *__restrict__ cval, const int32_t *__restrict__ rowptrX, const int32_t *__restrict__ colX,         \
      const T *__restrict__ valX, const T *__restrict__ q, const T *__restrict__ e, const V4<T> *m, T *uw
#define PMFEM_PRECORR_BODY                                                                                      \
  extern __shared__ __align__(16) unsigned char pipe_raw[];                                                    \
  pdl_enter();                                                                                                  \
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;                                            \
  if (t >= Np) return;                                                                                          \
  const int64_t i = map ? (int64_t)map[t] : t;                                                                  \
  precorr_row<T, CT, VT, cor_pipe<VT>()>(t, i, 0, (int32_t)Np, clen, cbase, coff, dcol, cval, rowptrX, colX,   \
                                         valX, q, e, m, uw,                                                     \
                                         pipe_raw + (threadIdx.x >> 5) * (cor_pipe<VT>() * PipeStage<VT, CT>::BYTES));
template <typename T, typename CT, typename VT>
__global__ void __launch_bounds__(kBlock, PMFEM_INTERP_MINB) k_precorr_capped(PMFEM_PRECORR_PARAMS) {
  PMFEM_PRECORR_BODY
}
template <typename T, typename CT, typename VT>
__global__ void __launch_bounds__(kBlock) k_precorr(PMFEM_PRECORR_PARAMS) {
  PMFEM_PRECORR_BODY
}
#undef PMFEM_PRECORR_BODY
#undef PMFEM_PRECORR_PARAMS
template <typename T, typename CT, typename VT>
constexpr auto precorr_kernel() {
  if constexpr (sizeof(T) == 4)
    return k_precorr_capped<T, CT, VT>;
  else
    return k_precorr<T, CT, VT>;
}

// PMFEM_STENCIL_MINB: optional register cap of the stencil pass (measured: 6 blocks per SM,
// 40 registers, no faster than the compiler's choice, so unset by default)
#ifdef PMFEM_STENCIL_MINB
#define PMFEM_STENCIL_LB __launch_bounds__(kBlock, PMFEM_STENCIL_MINB)
#else
#define PMFEM_STENCIL_LB __launch_bounds__(kBlock)
#endif
template <typename T, int P>
__global__ void PMFEM_STENCIL_LB k_stencil(int64_t Np, const int32_t* __restrict__ base,
                                                   const T* __restrict__ frac, const T* __restrict__ U, int N0,
                                                   int N1, int N2, bool p0, bool p1, bool p2, T* uw) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  stencil_add_row<T, P>(i, base, frac, U, N0, N1, N2, p0, p1, p2, uw);
}

// ---------------------------------------------------------------- gradient + exchange + RK4
// Two instances of the same body: with FP32 operator values the kernel asks for
// PMFEM_FIELD_MINB resident blocks per SM (a register cap: measured 78 -> 72 us on the 1M-node
// wire); with bfloat16 values (the cap measured 59 -> 62 us there) and FP64 the compiler chooses.
#ifndef PMFEM_FIELD_MINB
#define PMFEM_FIELD_MINB 5
#endif
#define PMFEM_FIELD_PARAMS                                                                                      \
  int64_t Np, const int32_t *__restrict__ len, const int32_t *__restrict__ base, const int64_t *__restrict__ off, \
      const CT *__restrict__ dcol, const VG *__restrict__ gx, const VG *__restrict__ gy,                          \
      const VG *__restrict__ gz, const VK *__restrict__ kp, const V4<T> *__restrict__ m,                          \
      const int32_t *__restrict__ perm, T *__restrict__ H, int use_ms, int use_ex, T hx, T hy, T hz,             \
      V4<T> *__restrict__ m0, V4<T> *__restrict__ mnext, V4<T> *__restrict__ accb, T cdt, T bw, int acc_init,    \
      T dt6, T gam, T alpha, int *flag, LocalTerms<T> lt
#define PMFEM_FIELD_BODY                                                                                        \
  pdl_enter();                                                                                                  \
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;                                            \
  if (i >= Np) return;                                                                                          \
  const int64_t uo = MODE == 0 ? (int64_t)perm[i] : 0;                                                          \
  field_row<T, MODE, CT, VG, VK, LOC>(i, 0, (int32_t)Np, len, base, off, dcol, gx, gy, gz, kp, m, uo, H, use_ms, \
                                      use_ex, hx, hy, hz, m0, mnext, accb, cdt, bw, acc_init, dt6, gam, alpha, flag, \
                                      lt);
template <typename T, int MODE, typename CT, typename VG, typename VK, bool LOC>
__global__ void __launch_bounds__(kBlock, PMFEM_FIELD_MINB) k_field_capped(PMFEM_FIELD_PARAMS) {
  PMFEM_FIELD_BODY
}
template <typename T, int MODE, typename CT, typename VG, typename VK, bool LOC>
__global__ void __launch_bounds__(kBlock) k_field(PMFEM_FIELD_PARAMS) {
  PMFEM_FIELD_BODY
}
#undef PMFEM_FIELD_BODY
#undef PMFEM_FIELD_PARAMS
template <typename T, int MODE, typename CT, typename VG, typename VK, bool LOC>
constexpr auto field_kernel() {
  if constexpr (sizeof(T) == 4 && sizeof(VG) == 4 && sizeof(VK) == 4)
    return k_field_capped<T, MODE, CT, VG, VK, LOC>;
  else
    return k_field<T, MODE, CT, VG, VK, LOC>;
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

// Launch-time choice of the column delta type and of the stored value type: f is called
// with Tag<int16_t> / Tag<int32_t>, and with Tag<T> or (FP32 arithmetic only) Tag<bf16_t>.
template <typename X>
struct Tag {
  using type = X;
};
template <typename T, typename F>
void with_ct(const DevSell<T>& M, F&& f) {
  if (M.col16)
    f(Tag<int16_t>{});
  else
    f(Tag<int32_t>{});
}
template <typename T, typename F>
void with_vt(bool bf, F&& f) {
  if constexpr (sizeof(T) == 4) {
    if (bf) {
      f(Tag<bf16_t>{});
      return;
    }
  }
  f(Tag<T>{});
}
template <typename VT, typename T>
const VT* vals(const DevSell<T>& M, int c) {
  return M.bval[c] ? (const VT*)(const void*)M.bval[c] : (const VT*)(const void*)M.val[c];
}

template <typename T>
void launch_charges(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const DevSell<T>& A = d.adj;
  d.prof.begin(KID_CHARGES, st);
  with_ct(A, [&](auto ct) {
    using CT = typename decltype(ct)::type;
    with_vt<T>(A.bval[0] != nullptr, [&](auto vt) {
      using VT = typename decltype(vt)::type;
      launch_k(k_charges<T, CT, VT>, blocks_for(d.Np), kBlock, 0, st, 
          d.Np, A.len, A.base, A.off, (const CT*)A.delta, vals<VT>(A, 0), vals<VT>(A, 1), vals<VT>(A, 2),
          vals<VT>(A, 3), vals<VT>(A, 4), vals<VT>(A, 5), m, d.q, d.e);
    });
  });
  d.prof.end(KID_CHARGES, st);
}

template <typename T>
void launch_anterp(const DevOps<T>& d, cudaStream_t st) {
  const DevSell<T>& Pm = d.pro;
  d.prof.begin(KID_ANTERP, st);
  // an operator that holds only the grid points some node projects to: clear the grid first
  const int64_t G = Pm.rows, Ggrid = (int64_t)d.dims[0] * d.dims[1] * d.dims[2];
  if (G < Ggrid) cudaMemsetAsync(d.grid, 0, (size_t)Ggrid * sizeof(T), st);
  if (G > 0)
    with_ct(Pm, [&](auto ct) {
      using CT = typename decltype(ct)::type;
      with_vt<T>(Pm.bval[0] != nullptr, [&](auto vt) {
        using VT = typename decltype(vt)::type;
        launch_k(k_project<T, CT, VT>, blocks_for(G), kBlock, 0, st, G, d.Np, Pm.map, Pm.len, Pm.base, Pm.off,
                                                                (const CT*)Pm.delta, vals<VT>(Pm, 0), d.q, d.grid);
      });
    });
  if (d.nx_exc > 0)
    launch_k(k_project_exc<T>, blocks_for(d.nx_exc), kBlock, 0, st, d.nx_exc, d.xnode, d.xgrid, d.xw, d.q, d.grid);
  d.prof.end(KID_ANTERP, st);
}

template <typename T>
void launch_interp(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np);
  const DevSell<T>& C = d.cor;
  d.prof.begin(KID_INTERP, st);
  with_ct(C, [&](auto ct) {
    using CT = typename decltype(ct)::type;
    with_vt<T>(C.bval[0] != nullptr, [&](auto vt) {
      using VT = typename decltype(vt)::type;
      const size_t sm = (size_t)(kBlock / 32) * cor_pipe<VT>() * PipeStage<VT, CT>::BYTES;
      auto go = [&](auto kernel) {
        set_smem(kernel, sm);
        launch_k(kernel, nb, kBlock, sm, st, d.Np, C.map, d.base, d.frac, d.grid, d.dims[0], d.dims[1], d.dims[2],
                                      d.periodic[0], d.periodic[1], d.periodic[2], C.len, C.base, C.off,
                                      (const CT*)C.delta, vals<VT>(C, 0), d.rowptrX, d.colX, d.valX, d.q, d.e, m,
                                      reinterpret_cast<T*>(const_cast<V4<T>*>(m)) + 3);   // u -> lane 3 of m
      };
      switch (d.p) {
        case 2: go(interp_kernel<T, 3, CT, VT>()); break;
        case 3: go(interp_kernel<T, 4, CT, VT>()); break;
        case 4: go(interp_kernel<T, 5, CT, VT>()); break;
        default: go(interp_kernel<T, 6, CT, VT>()); break;
      }
    });
  });
  d.prof.end(KID_INTERP, st);
}

template <typename T>
void launch_precorr(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np);
  const DevSell<T>& C = d.cor;
  d.prof.begin(KID_INTERP, st);
  with_ct(C, [&](auto ct) {
    using CT = typename decltype(ct)::type;
    with_vt<T>(C.bval[0] != nullptr, [&](auto vt) {
      using VT = typename decltype(vt)::type;
      const size_t sm = (size_t)(kBlock / 32) * cor_pipe<VT>() * PipeStage<VT, CT>::BYTES;
      auto kernel = precorr_kernel<T, CT, VT>();
      set_smem(kernel, sm);
      kernel<<<nb, kBlock, sm, st>>>(d.Np, C.map, C.len, C.base, C.off, (const CT*)C.delta, vals<VT>(C, 0),
                                    d.rowptrX, d.colX, d.valX, d.q, d.e, m,
                                    reinterpret_cast<T*>(const_cast<V4<T>*>(m)) + 3);   // u -> lane 3 of m
    });
  });
  d.prof.end(KID_INTERP, st);
}

template <typename T>
void launch_stencil(const DevOps<T>& d, const V4<T>* m, cudaStream_t st) {
  const unsigned nb = blocks_for(d.Np);
  T* uw = reinterpret_cast<T*>(const_cast<V4<T>*>(m)) + 3;
  d.prof.begin(KID_STENCIL, st);
  auto go = [&](auto kernel) {
    launch_k(kernel, nb, kBlock, 0, st, d.Np, d.base, d.frac, d.grid, d.dims[0], d.dims[1], d.dims[2], d.periodic[0],
                                  d.periodic[1], d.periodic[2], uw);
  };
  switch (d.p) {
    case 2: go(k_stencil<T, 3>); break;
    case 3: go(k_stencil<T, 4>); break;
    case 4: go(k_stencil<T, 5>); break;
    default: go(k_stencil<T, 6>); break;
  }
  d.prof.end(KID_STENCIL, st);
}

template <typename T>
void launch_field(const DevOps<T>& d, const V4<T>* m, T* H, int comps, double hx, double hy, double hz,
                  const RkArgs& rk, cudaStream_t st) {
  const DevSell<T>& A = d.adj;
  const unsigned nb = blocks_for(d.Np);
  const int use_ms = (comps & 2) ? 1 : 0, use_ex = (comps & 1) ? 1 : 0;
  const bool loc = (comps & 8) && d.loc.ptr;
  const T ax = (comps & 4) ? (T)hx : T(0), ay = (comps & 4) ? (T)hy : T(0), az = (comps & 4) ? (T)hz : T(0);
  V4<T>* m0 = (V4<T>*)rk.m0;
  V4<T>* mn = (V4<T>*)rk.mnext;
  V4<T>* acc = (V4<T>*)rk.acc;
  d.prof.begin(KID_FIELD, st);
  with_ct(A, [&](auto ct) {
    using CT = typename decltype(ct)::type;
    with_vt<T>(A.bval[6] != nullptr, [&](auto vg) {
      using VG = typename decltype(vg)::type;
      with_vt<T>(A.bval[9] != nullptr, [&](auto vk) {
        using VK = typename decltype(vk)::type;
        auto go = [&](auto kernel) {
          launch_k(kernel, nb, kBlock, 0, st, d.Np, A.len, A.base, A.off, (const CT*)A.delta, vals<VG>(A, 6),
                                        vals<VG>(A, 7), vals<VG>(A, 8), vals<VK>(A, 9), m, d.perm, H, use_ms,
                                        use_ex, ax, ay, az, m0, mn, acc, (T)rk.cdt, (T)rk.bw, rk.acc_init,
                                        (T)rk.dt6, (T)rk.gam, (T)rk.alpha, d.flag, d.loc);
        };
        if (loc) {
          if (rk.mode == 0)
            go(field_kernel<T, 0, CT, VG, VK, true>());
          else if (rk.mode == 1)
            go(field_kernel<T, 1, CT, VG, VK, true>());
          else
            go(field_kernel<T, 2, CT, VG, VK, true>());
        } else if (rk.mode == 0) {
          go(field_kernel<T, 0, CT, VG, VK, false>());
        } else if (rk.mode == 1) {
          go(field_kernel<T, 1, CT, VG, VK, false>());
        } else {
          go(field_kernel<T, 2, CT, VG, VK, false>());
        }
      });
    });
  });
  d.prof.end(KID_FIELD, st);
}

// ---------------------------------------------------------------- layout checks
namespace {
template <typename CT>
__global__ void k_check_sell(int64_t rows, int64_t map_lim, int64_t ncols, int vw, const int32_t* __restrict__ map,
                             const int32_t* __restrict__ len, const int32_t* __restrict__ base,
                             const int64_t* __restrict__ off, const CT* __restrict__ dcol, int* flag) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows) return;
  bool bad = false;
  if (map && (map[t] < 0 || map[t] >= map_lim)) bad = true;
  const int64_t c = t >> 5, lane = t & 31;
  const int64_t width = (off[c + 1] - off[c]) / 32;   // padded entries per lane of this chunk
  const int32_t n = len[t], b = base[t];
  if (n < 0 || n > width || (n > 0 && (b < 0 || b >= ncols))) bad = true;
  for (int32_t j = 0; j < n && !bad; ++j) {
    const int64_t o = off[c] + ((int64_t)(j / vw) * 32 + lane) * vw + j % vw;
    const int64_t d = (int64_t)dcol[o];
    if (d <= -ncols || d >= ncols) bad = true;
  }
  if (bad) atomicOr(flag, FLAG_LAYOUT);
}

// stencil bases inside the grid along open axes (so the stencil passes stay in the grid)
__global__ void k_check_stencils(int64_t Np, const int32_t* __restrict__ base, int N0, int N1, int N2, int p0, int p1,
                                 int p2, int P, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Np) return;
  const int Nn[3] = {N0, N1, N2}, pp[3] = {p0, p1, p2};
  bool bad = false;
  for (int a = 0; a < 3; ++a)
    if (!pp[a] && (base[3 * i + a] < 0 || base[3 * i + a] + P > Nn[a])) bad = true;
  if (bad) atomicOr(flag, FLAG_LAYOUT);
}

// projection exceptions: node and grid indices in range
__global__ void k_check_exceptions(int64_t n, int64_t Np, int64_t G, const int32_t* __restrict__ node,
                                   const int64_t* __restrict__ gidx, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (node[i] < 0 || node[i] >= Np || gidx[i] < 0 || gidx[i] >= G) atomicOr(flag, FLAG_LAYOUT);
}

// map_lim: the rows the map points into (the operator's own rows, or the grid points for the
// projection, whose rows are only the grid points with entries)
template <typename T>
void check_sell(const DevSell<T>& M, int64_t map_lim, int64_t ncols, int vw, int* flag, cudaStream_t st) {
  if (M.rows <= 0) return;
  if (M.col16)
    k_check_sell<int16_t><<<blocks_for(M.rows), kBlock, 0, st>>>(M.rows, map_lim, ncols, vw, M.map, M.len, M.base,
                                                                  M.off, (const int16_t*)M.delta, flag);
  else
    k_check_sell<int32_t><<<blocks_for(M.rows), kBlock, 0, st>>>(M.rows, map_lim, ncols, vw, M.map, M.len, M.base,
                                                                  M.off, (const int32_t*)M.delta, flag);
}
}  // namespace

template <typename T>
void launch_layout_checks(const DevOps<T>& d, cudaStream_t st) {
  check_sell(d.adj, d.adj.rows, d.Np, 4, d.flag, st);
  check_sell(d.cor, d.cor.rows, d.Np, PMFEM_COR_VW, d.flag, st);
  check_sell(d.pro, (int64_t)d.dims[0] * d.dims[1] * d.dims[2], d.Np, PMFEM_COR_VW, d.flag, st);
  if (d.Np > 0)
    k_check_stencils<<<blocks_for(d.Np), kBlock, 0, st>>>(d.Np, d.base, d.dims[0], d.dims[1], d.dims[2],
                                                        d.periodic[0] ? 1 : 0, d.periodic[1] ? 1 : 0,
                                                        d.periodic[2] ? 1 : 0, d.p + 1, d.flag);
  if (d.nx_exc > 0)
    k_check_exceptions<<<blocks_for(d.nx_exc), kBlock, 0, st>>>(d.nx_exc, d.Np,
                                                                 (int64_t)d.dims[0] * d.dims[1] * d.dims[2],
                                                                 d.xnode, d.xgrid, d.flag);
}

#define PMFEM_INSTANTIATE(T)                                                                          \
  template void launch_layout_checks<T>(const DevOps<T>&, cudaStream_t);                             \
  template void launch_perm_in<T>(const DevOps<T>&, const T*, V4<T>*, cudaStream_t);                 \
  template void launch_perm_out<T>(const DevOps<T>&, const V4<T>*, T*, cudaStream_t);                \
  template void launch_charges<T>(const DevOps<T>&, const V4<T>*, cudaStream_t);                     \
  template void launch_anterp<T>(const DevOps<T>&, cudaStream_t);                                    \
  template void launch_interp<T>(const DevOps<T>&, const V4<T>*, cudaStream_t);                      \
  template void launch_precorr<T>(const DevOps<T>&, const V4<T>*, cudaStream_t);                     \
  template void launch_stencil<T>(const DevOps<T>&, const V4<T>*, cudaStream_t);                     \
  template void launch_field<T>(const DevOps<T>&, const V4<T>*, T*, int, double, double, double, const RkArgs&, \
                                cudaStream_t);
PMFEM_INSTANTIATE(double)
PMFEM_INSTANTIATE(float)
#undef PMFEM_INSTANTIATE

}  // namespace pmfem
