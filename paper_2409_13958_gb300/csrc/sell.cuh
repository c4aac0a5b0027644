// Device building blocks shared by the single-mesh kernels (kernels.cu) and the batched
// kernels (batch.cu): Lagrange weights, periodic wrap, SELL-32 column decoding and value
// loads, and one row of each sparse pass.  A row function works on global indices; the
// caller gives the column origin c0 and the column count nc of the row's mesh, so that a
// column is c0 + ((base + delta) mod nc).  A single mesh uses c0 = 0, nc = N'.
#pragma once

#include <cmath>

#include "device.hpp"

namespace pmfem {
namespace {

constexpr int kBlock = 256;

// values of a precorrection row each lane keeps in flight: 4 x PMFEM_COR_G (vector width 4), or
// 8 x (PMFEM_COR_G + 1) / 2 (vector width 8)
#ifndef PMFEM_COR_G
#define PMFEM_COR_G 4
#endif
// groups of 8 projection entries each lane keeps in flight (rows are short: about two groups;
// two in flight measured no faster than one)
#ifndef PMFEM_PRO_G
#define PMFEM_PRO_G 1
#endif

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// prod_{j != a} (a - j): the denominator of Lagrange basis polynomial a of the nodes 0 .. P-1
// (an integer of magnitude at most 5! for P <= 6)
template <int P>
__host__ __device__ constexpr double lagrange_den(int a) {
  double d = 1.0;
  for (int j = 0; j < P; ++j)
    if (j != a) d *= (double)(a - j);
  return d;
}

// The P Lagrange basis polynomials of the nodes 0 .. P-1 at s: the product of (s - j) over
// j != a times the compile-time reciprocal of its denominator (no division at run time).
template <typename T, int P>
__device__ __forceinline__ void lagrange(T s, T (&w)[P]) {
#pragma unroll
  for (int i = 0; i < P; ++i) {
    T v = T(1);
#pragma unroll
    for (int j = 0; j < P; ++j)
      if (j != i) v *= (s - T(j));
    w[i] = v * T(1.0 / lagrange_den<P>(i));
  }
}

__device__ __forceinline__ int wrap(int i, int N, bool per) {
  if (per) {
    if (i < 0) i += N;
    if (i >= N) i -= N;
  }
  return i;
}

// Column of a SELL entry: the row's base plus the stored delta, modulo the number of
// columns n (deltas are stored modulo n, so a row that straddles the periodic seam of the
// box order keeps small deltas).  b is in [0, n) and |d| <= n/2 with n <= 2^30 (checked
// when the mesh is created), so b + d fits in int32 and one correction suffices.
template <typename CT>
__device__ __forceinline__ int32_t col_of(int32_t b, CT d, int32_t n) {
  int32_t c = b + (int32_t)d;
  c = c < 0 ? c + n : c;
  c = c >= n ? c - n : c;
#if defined(PMFEM_CHECKS) && PMFEM_CHECKS
  c = (c < 0 || c >= n) ? 0 : c;   // checked builds never gather outside the vector (the layout
                                   // checks report the bad index at upload)
#endif
  return c;
}

// Streaming load of a stored operator value, widened to the arithmetic type T.  Values are
// stored as T, or (BF16-split precision) as the upper 16 bits of an FP32 number (bfloat16),
// which widen exactly by a shift.
template <typename T>
__device__ __forceinline__ T ldv(const T* p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ T ldv(const bf16_t* p) {
  return __uint_as_float((uint32_t)__ldcs(&p->bits) << 16);
}

// sum_j val[o_j] * x[col(b, delta[o_j])] over one SELL row, o_j = o + 32 j: the value and
// column loads of a batch of B elements are issued together, then their B gathers, so
// each thread keeps 2B independent loads in flight instead of one dependent pair.  The
// remainder loop is left to the compiler, which unrolls it (a loop kept rolled there
// serialises up to B - 1 dependent load pairs per row).
template <int B, typename T, typename CT, typename VT>
__device__ __forceinline__ T sell_dot(const VT* __restrict__ val, const CT* __restrict__ dcol,
                                      const T* __restrict__ x, int32_t b, int64_t o, int n, int32_t ncol) {
  T acc = 0;
  int j = 0;
  for (; j + B <= n; j += B, o += 32 * B) {
    T v[B];
    int32_t c[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      v[k] = ldv<T>(val + o + 32 * k);
      c[k] = col_of(b, __ldcs(dcol + o + 32 * k), ncol);
    }
#pragma unroll
    for (int k = 0; k < B; ++k) acc += v[k] * __ldg(x + c[k]);
  }
  for (; j < n; ++j, o += 32) acc += ldv<T>(val + o) * __ldg(x + col_of(b, __ldcs(dcol + o), ncol));
  return acc;
}

// Loads of the operator streams (values and column deltas, each read once per evaluation).
// PMFEM_STREAM_LD 0: ld.global.cs (evict-first in L1 and L2); 1: ld.global.nc with
// L1::no_allocate, which leaves L1 to the gathers of x; 2: as 1, and 32-byte loads also
// evict-first in L2.  With W = true the 32 bytes of a lane's step (8 FP32 values, 8 int32
// deltas, 4 FP64 values) come in one 256-bit load (measured: -4% for the precorrection,
// -25% for the FP64 projection, +5% for the FP32 projection, whose rows are short); every
// chunk offset is a multiple of the vector width (checked at upload), so these addresses are
// 32-byte aligned.  PMFEM_LD256 0 turns the 256-bit loads off everywhere.
#ifndef PMFEM_STREAM_LD
#define PMFEM_STREAM_LD 0
#endif
#ifndef PMFEM_LD256
#define PMFEM_LD256 1
#endif
__device__ __forceinline__ uint4 lds_16(const void* p) {
#if PMFEM_STREAM_LD == 0
  return __ldcs(reinterpret_cast<const uint4*>(p));
#else
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
#endif
}
__device__ __forceinline__ uint2 lds_8(const void* p) {
#if PMFEM_STREAM_LD == 0
  return __ldcs(reinterpret_cast<const uint2*>(p));
#else
  uint2 r;
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
#endif
}
template <bool W = true>
__device__ __forceinline__ void lds_32(const void* p, uint32_t (&r)[8]) {
  if constexpr (W && PMFEM_LD256) {
#if PMFEM_STREAM_LD == 0
#define PMFEM_LD256_OP "ld.global.cs.v8.b32"
#elif PMFEM_STREAM_LD == 1
#define PMFEM_LD256_OP "ld.global.nc.L1::no_allocate.v8.b32"
#else
#define PMFEM_LD256_OP "ld.global.nc.L1::no_allocate.L2::evict_first.v8.b32"
#endif
    asm(PMFEM_LD256_OP " {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
#undef PMFEM_LD256_OP
  } else {
    const uint4 a = lds_16(p), b = lds_16(static_cast<const char*>(p) + 16);
    r[0] = a.x, r[1] = a.y, r[2] = a.z, r[3] = a.w, r[4] = b.x, r[5] = b.y, r[6] = b.z, r[7] = b.w;
  }
}
__device__ __forceinline__ double dbl(uint32_t lo, uint32_t hi) { return __hiloint2double((int)hi, (int)lo); }

// Four consecutive stored values of one lane (16 B of FP32, 32 B of FP64, 8 B of bfloat16),
// widened to T, and four consecutive column deltas (8 B of int16 or 16 B of int32).
__device__ __forceinline__ void ldv4(const float* p, float (&v)[4]) {
  const uint4 a = lds_16(p);
  v[0] = __uint_as_float(a.x), v[1] = __uint_as_float(a.y), v[2] = __uint_as_float(a.z), v[3] = __uint_as_float(a.w);
}
__device__ __forceinline__ void ldv4(const double* p, double (&v)[4]) {
  uint32_t r[8];
  lds_32(p, r);
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = dbl(r[2 * k], r[2 * k + 1]);
}
__device__ __forceinline__ void ldv4(const bf16_t* p, float (&v)[4]) {
  const uint2 a = lds_8(p);
  v[0] = __uint_as_float(a.x << 16), v[1] = __uint_as_float(a.x & 0xffff0000u);
  v[2] = __uint_as_float(a.y << 16), v[3] = __uint_as_float(a.y & 0xffff0000u);
}
__device__ __forceinline__ void ldc4(const int16_t* p, int32_t (&c)[4]) {
  const uint2 a = lds_8(p);
  c[0] = (int32_t)(int16_t)(a.x & 0xffffu), c[1] = (int32_t)(int16_t)(a.x >> 16);
  c[2] = (int32_t)(int16_t)(a.y & 0xffffu), c[3] = (int32_t)(int16_t)(a.y >> 16);
}
__device__ __forceinline__ void ldc4(const int32_t* p, int32_t (&c)[4]) {
  const uint4 a = lds_16(p);
  c[0] = (int32_t)a.x, c[1] = (int32_t)a.y, c[2] = (int32_t)a.z, c[3] = (int32_t)a.w;
}

template <bool W = true>
__device__ __forceinline__ void ldv8(const float* p, float (&v)[8]) {
  uint32_t r[8];
  lds_32<W>(p, r);
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
template <bool W = true>
__device__ __forceinline__ void ldv8(const double* p, double (&v)[8]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t r[8];
    lds_32<W>(p + 4 * h, r);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[4 * h + k] = dbl(r[2 * k], r[2 * k + 1]);
  }
}
template <bool W = true>
__device__ __forceinline__ void ldv8(const bf16_t* p, float (&v)[8]) {
  const uint4 a = lds_16(p);
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) v[2 * k] = __uint_as_float(w[k] << 16), v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
}
template <bool W = true>
__device__ __forceinline__ void ldc8(const int16_t* p, int32_t (&c)[8]) {
  const uint4 a = lds_16(p);
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) c[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu), c[2 * k + 1] = (int32_t)(int16_t)(w[k] >> 16);
}
template <bool W = true>
__device__ __forceinline__ void ldc8(const int32_t* p, int32_t (&c)[8]) {
  uint32_t r[8];
  lds_32<W>(p, r);
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = (int32_t)r[k];
}

// sell_dot for a SELL-32 operator stored eight values per lane and step (vector width 8):
// group g of the lane at o0 + 256 g with o0 = off[c] + 8 lane; rows padded to whole groups
// with value 0 and delta 0 (a valid column), so every group is read whole.
template <int G, bool W = true, typename T, typename CT, typename VT>
__device__ __forceinline__ T sell_dot8(const VT* __restrict__ val, const CT* __restrict__ dcol,
                                       const T* __restrict__ x, int32_t b, int64_t o0, int n, int32_t ncol) {
  T acc = 0;
  const int ng = (n + 7) >> 3;
  int g = 0;
  for (; g + G <= ng; g += G, o0 += 256 * G) {
    T v[G][8];
    int32_t c[G][8];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      ldv8<W>(val + o0 + 256 * k, v[k]);
      ldc8<W>(dcol + o0 + 256 * k, c[k]);
    }
#pragma unroll
    for (int k = 0; k < G; ++k)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc += v[k][e] * __ldg(x + col_of(b, c[k][e], ncol));
  }
  for (; g < ng; ++g, o0 += 256) {
    T v[8];
    int32_t c[8];
    ldv8<W>(val + o0, v);
    ldc8<W>(dcol + o0, c);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc += v[e] * __ldg(x + col_of(b, c[e], ncol));
  }
  return acc;
}

// Pipelined form of sell_dot8: each lane streams its own groups into shared memory with
// 16-byte cp.async copies, S - 1 groups ahead of the one it multiplies, so the DRAM latency
// of the value and delta streams overlaps the gathers of x instead of holding registers.
// buf is the warp's buffer of S stages; a stage holds, for each of the 32 lanes, the lane's
// 8 values and 8 deltas as 16-byte pieces, piece k of lane l at (32 k + l) x 16 bytes (eight
// consecutive lanes read 128 contiguous bytes: no bank conflicts).  A lane reads only the
// pieces it copied itself, so no barrier is needed; cp.async.wait_group orders them.
template <typename VT, typename CT>
struct PipeStage {
  static constexpr int PV = 8 * (int)sizeof(VT) / 16;   // 16-byte pieces of values
  static constexpr int PC = 8 * (int)sizeof(CT) / 16;   // 16-byte pieces of deltas
  static constexpr int BYTES = 32 * 16 * (PV + PC);      // one stage of one warp
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint4 lds16(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void unpack8(const uint4 (&w)[2], float (&v)[8]) {
  const uint32_t a[8] = {w[0].x, w[0].y, w[0].z, w[0].w, w[1].x, w[1].y, w[1].z, w[1].w};
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(a[k]);
}
__device__ __forceinline__ void unpack8(const uint4 (&w)[4], double (&v)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = __hiloint2double((int)w[k].y, (int)w[k].x);
    v[2 * k + 1] = __hiloint2double((int)w[k].w, (int)w[k].z);
  }
}
__device__ __forceinline__ void unpack8(const uint4 (&w)[1], float (&v)[8]) {   // bfloat16
  const uint32_t a[4] = {w[0].x, w[0].y, w[0].z, w[0].w};
#pragma unroll
  for (int k = 0; k < 4; ++k) v[2 * k] = __uint_as_float(a[k] << 16), v[2 * k + 1] = __uint_as_float(a[k] & 0xffff0000u);
}
__device__ __forceinline__ void unpackc8(const uint4 (&w)[1], int32_t (&c)[8]) {   // int16 deltas
  const uint32_t a[4] = {w[0].x, w[0].y, w[0].z, w[0].w};
#pragma unroll
  for (int k = 0; k < 4; ++k) c[2 * k] = (int32_t)(int16_t)(a[k] & 0xffffu), c[2 * k + 1] = (int32_t)(int16_t)(a[k] >> 16);
}
__device__ __forceinline__ void unpackc8(const uint4 (&w)[2], int32_t (&c)[8]) {   // int32 deltas
  const uint32_t a[8] = {w[0].x, w[0].y, w[0].z, w[0].w, w[1].x, w[1].y, w[1].z, w[1].w};
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = (int32_t)a[k];
}

template <int S, typename T, typename CT, typename VT>
__device__ __forceinline__ T sell_dot8_pipe(const VT* __restrict__ val, const CT* __restrict__ dcol,
                                            const T* __restrict__ x, int32_t b, int64_t o0, int n, int32_t ncol,
                                            unsigned char* buf) {
  using PS = PipeStage<VT, CT>;
  const int lane = threadIdx.x & 31;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(buf) + 16u * (uint32_t)lane;
  const int ng = (n + 7) >> 3;
  auto issue = [&](int g, int slot) {
    const uint32_t s = s0 + (uint32_t)(slot * PS::BYTES);
    const char* pv = reinterpret_cast<const char*>(val + o0 + 256 * (int64_t)g);
    const char* pc = reinterpret_cast<const char*>(dcol + o0 + 256 * (int64_t)g);
#pragma unroll
    for (int k = 0; k < PS::PV; ++k) cp_async16(s + 512u * k, pv + 16 * k);
#pragma unroll
    for (int k = 0; k < PS::PC; ++k) cp_async16(s + 512u * (PS::PV + k), pc + 16 * k);
  };
#pragma unroll
  for (int g = 0; g < S - 1; ++g) {
    if (g < ng) issue(g, g);
    cp_async_commit();
  }
  T acc = 0;
  int slot = 0;                       // slot of group g; group g + S - 1 goes to the slot of g - 1
  for (int g = 0; g < ng; ++g) {
    const int fill = slot == 0 ? S - 1 : slot - 1;
    if (g + S - 1 < ng) issue(g + S - 1, fill);
    cp_async_commit();
    cp_async_wait<S - 1>();
    const uint32_t s = s0 + (uint32_t)(slot * PS::BYTES);
    uint4 wv[PS::PV], wc[PS::PC];
#pragma unroll
    for (int k = 0; k < PS::PV; ++k) wv[k] = lds16(s + 512u * k);
#pragma unroll
    for (int k = 0; k < PS::PC; ++k) wc[k] = lds16(s + 512u * (PS::PV + k));
    T v[8];
    int32_t c[8];
    unpack8(wv, v);
    unpackc8(wc, c);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc += v[e] * __ldg(x + col_of(b, c[e], ncol));
    slot = slot == S - 1 ? 0 : slot + 1;
  }
  return acc;
}

// sell_dot for a SELL-32 operator stored four values per lane and step (vector width 4):
// the lane's group g of elements 4g .. 4g+3 sits at o0 + 128 g, where o0 = off[c] + 4 lane.
// Rows are padded to whole groups with value 0 and delta 0 (a valid column), so every group
// is read whole; G groups (4G values, 4G deltas, then 4G gathers) are kept in flight.
template <int G, typename T, typename CT, typename VT>
__device__ __forceinline__ T sell_dot4(const VT* __restrict__ val, const CT* __restrict__ dcol,
                                       const T* __restrict__ x, int32_t b, int64_t o0, int n, int32_t ncol) {
  T acc = 0;
  const int ng = (n + 3) >> 2;
  int g = 0;
  for (; g + G <= ng; g += G, o0 += 128 * G) {
    T v[G][4];
    int32_t c[G][4];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      ldv4(val + o0 + 128 * k, v[k]);
      ldc4(dcol + o0 + 128 * k, c[k]);
    }
#pragma unroll
    for (int k = 0; k < G; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc += v[k][e] * __ldg(x + col_of(b, c[k][e], ncol));
  }
  for (; g < ng; ++g, o0 += 128) {
    T v[4];
    int32_t c[4];
    ldv4(val + o0, v);
    ldc4(dcol + o0, c);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc += v[e] * __ldg(x + col_of(b, c[e], ncol));
  }
  return acc;
}

// ---------------------------------------------------------------- charges
// q = W^q M (Eq. 14a) and e = E M (touching-element part of Eq. 14c): adjacency row i, stored
// with vector width 4 (group g of the row at off[c] + 4 lane + 128 g; padded with zeros).
template <typename T, typename CT, typename VT>
__device__ __forceinline__ void charges_row(int64_t i, int64_t c0, int32_t nc, const int32_t* __restrict__ len,
                                            const int32_t* __restrict__ base, const int64_t* __restrict__ off,
                                            const CT* __restrict__ dcol, const VT* __restrict__ wx,
                                            const VT* __restrict__ wy, const VT* __restrict__ wz,
                                            const VT* __restrict__ ex, const VT* __restrict__ ey,
                                            const VT* __restrict__ ez, const V4<T>* __restrict__ m,
                                            T* __restrict__ q, T* __restrict__ e) {
  const int ng = (len[i] + 3) >> 2;
  int64_t o = off[i >> 5] + 4 * (i & 31);
  const int32_t b = base[i];
  const V4<T>* mc = m + c0;
  T aq = 0, ae = 0;
  for (int g = 0; g < ng; ++g, o += 128) {
    int32_t c[4];
    T a0[4], a1[4], a2[4], e0[4], e1[4], e2[4];
    ldc4(dcol + o, c);
    ldv4(wx + o, a0);
    ldv4(wy + o, a1);
    ldv4(wz + o, a2);
    ldv4(ex + o, e0);
    ldv4(ey + o, e1);
    ldv4(ez + o, e2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const V4<T> mk = mc[col_of(b, c[k], nc)];
      aq += a0[k] * mk.x + a1[k] * mk.y + a2[k] * mk.z;
      ae += e0[k] * mk.x + e1[k] * mk.y + e2[k] * mk.z;
    }
  }
  q[i] = aq;
  e[i] = ae;
}

// ---------------------------------------------------------------- projection (step 1)
// Q = P^T q as a gather: grid point g (SELL row t) sums w q over the nodes whose stencil
// covers it (the nodes of the boxes [g - pr, g + pl] per axis, enumerated at set-up).
template <typename T, typename CT, typename VT>
__device__ __forceinline__ void project_row(int64_t t, int64_t g, int64_t c0, int32_t nc,
                                            const int32_t* __restrict__ len, const int32_t* __restrict__ base,
                                            const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                            const VT* __restrict__ pw, const T* __restrict__ q,
                                            T* __restrict__ grid) {
  const int n = len[t];
  T acc = 0;
  if (n > 0) {
    if constexpr (PMFEM_COR_VW == 8)
      acc = sell_dot8<PMFEM_PRO_G, sizeof(T) == 8>(pw, dcol, q + c0, base[t], off[t >> 5] + 8 * (t & 31), n, nc);
    else
      acc = sell_dot4<2>(pw, dcol, q + c0, base[t], off[t >> 5] + 4 * (t & 31), n, nc);
  }
  grid[g] = acc;
}

// ---------------------------------------------------------------- interpolation + precorrection
// Step 3 for node i: the (p+1)^3 Lagrange stencil over the grid potential U.
template <typename T, int P>
__device__ __forceinline__ T stencil_row(int64_t i, const int32_t* __restrict__ base, const T* __restrict__ frac,
                                         const T* __restrict__ U, int N0, int N1, int N2, bool p0, bool p1, bool p2) {
  T w0[P], w1[P], w2[P];
  lagrange<T, P>(frac[3 * i], w0);
  lagrange<T, P>(frac[3 * i + 1], w1);
  lagrange<T, P>(frac[3 * i + 2], w2);
  const int b0 = base[3 * i], b1 = base[3 * i + 1], b2 = base[3 * i + 2];
  T acc = 0;
  if constexpr (sizeof(T) == 4) {
    // FP32 grid, x taps inside one row (no periodic wrap along x): each row's P taps come from
    // the 16-byte-aligned chunks that hold them (one or two loads instead of P), weighted by the
    // x weights shifted to the taps' offset o within the first chunk.  A chunk is loaded only if
    // it holds a tap, so with N0 a multiple of 4 no load leaves the row.
    if (b0 >= 0 && b0 + P <= N0 && (N0 & 3) == 0) {
      constexpr int NCH = (P + 6) / 4;    // chunks that can hold taps o .. o + P - 1 for o < 4
      const int o = b0 & 3;
      const int nch = (o + P + 3) >> 2;   // chunks that do
      T ws[4 * NCH];
#pragma unroll
      for (int k = 0; k < 4 * NCH; ++k) {
        T v = 0;
#pragma unroll
        for (int a = 0; a < P; ++a) v = (k == o + a) ? w0[a] : v;
        ws[k] = v;
      }
#pragma unroll
      for (int c = 0; c < P; ++c) {
        const int64_t zo = (int64_t)N1 * wrap(b2 + c, N2, p2);
#pragma unroll
        for (int b = 0; b < P; ++b) {
          const float4* rowp = reinterpret_cast<const float4*>(U + (int64_t)N0 * (wrap(b1 + b, N1, p1) + zo) + (b0 - o));
          T s = 0;
#pragma unroll
          for (int h = 0; h < NCH; ++h) {
            if (h == 0 || h < nch) {
              const float4 v = __ldg(rowp + h);
              s += ws[4 * h] * v.x + ws[4 * h + 1] * v.y + ws[4 * h + 2] * v.z + ws[4 * h + 3] * v.w;
            }
          }
          acc += w2[c] * w1[b] * s;
        }
      }
      return acc;
    }
  }
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
  return acc;
}

// Near-element entries of node i beyond the adjacency pattern (CSR, 3-vector values on M).
template <typename T>
__device__ __forceinline__ T extras_row(int64_t i, const int32_t* __restrict__ rowptrX, const int32_t* __restrict__ colX,
                                        const T* __restrict__ valX, const V4<T>* m) {
  T acc = 0;
  for (int32_t p = rowptrX[i]; p < rowptrX[i + 1]; ++p) {
    const V4<T> mk = m[colX[p]];
    acc += valX[3 * p] * mk.x + valX[3 * p + 1] * mk.y + valX[3 * p + 2] * mk.z;
  }
  return acc;
}

// Potential of node i (SELL row t of the precorrection): the stencil (step 3), the point
// precorrection row (step 4), the near-element entries beyond the adjacency pattern and the
// touching-element part e.  The potential goes to the fourth (padding) lane of the node's
// magnetisation 4-vector, uw = (T*)m + 3, so that the gradient pass gathers m and u of a
// neighbour with one 16-byte load; this pass reads only the first three lanes of m.
// PIPE > 0 streams the precorrection row through the warp's PIPE-stage shared-memory buffer
// buf (sell_dot8_pipe; vector width 8 only); PIPE = 0 loads it into registers.
template <typename T, int P, typename CT, typename VT, int PIPE = 0>
__device__ __forceinline__ void interp_row(
    int64_t t, int64_t i, int64_t c0, int32_t nc, const int32_t* __restrict__ base, const T* __restrict__ frac,
    const T* __restrict__ U, int N0, int N1, int N2, bool p0, bool p1, bool p2, const int32_t* __restrict__ clen,
    const int32_t* __restrict__ cbase, const int64_t* __restrict__ coff, const CT* __restrict__ dcol,
    const VT* __restrict__ cval, const int32_t* __restrict__ rowptrX, const int32_t* __restrict__ colX,
    const T* __restrict__ valX, const T* __restrict__ q, const T* __restrict__ e, const V4<T>* m, T* uw,
    unsigned char* buf = nullptr) {
  T acc = stencil_row<T, P>(i, base, frac, U, N0, N1, N2, p0, p1, p2);
  if constexpr (PMFEM_COR_VW == 8 && PIPE > 0)
    acc += sell_dot8_pipe<PIPE>(cval, dcol, q + c0, cbase[t], coff[t >> 5] + 8 * (t & 31), clen[t], nc, buf);
  else if constexpr (PMFEM_COR_VW == 8)
    acc += sell_dot8<(PMFEM_COR_G + 1) / 2>(cval, dcol, q + c0, cbase[t], coff[t >> 5] + 8 * (t & 31), clen[t], nc);
  else
    acc += sell_dot4<PMFEM_COR_G>(cval, dcol, q + c0, cbase[t], coff[t >> 5] + 4 * (t & 31), clen[t], nc);
  acc += extras_row<T>(i, rowptrX, colX, valX, m);
  uw[4 * i] = acc + e[i];
}

// The same potential in two passes, so that the precorrection (which needs only q, m and e)
// can run while the projection and the FFT produce U: precorr_row writes the precorrection,
// near-element and touching-element parts to lane 3 of m; stencil_add_row then adds the
// stencil of U (step 3) for node i.
template <typename T, typename CT, typename VT, int PIPE = 0>
__device__ __forceinline__ void precorr_row(int64_t t, int64_t i, int64_t c0, int32_t nc,
                                            const int32_t* __restrict__ clen, const int32_t* __restrict__ cbase,
                                            const int64_t* __restrict__ coff, const CT* __restrict__ dcol,
                                            const VT* __restrict__ cval, const int32_t* __restrict__ rowptrX,
                                            const int32_t* __restrict__ colX, const T* __restrict__ valX,
                                            const T* __restrict__ q, const T* __restrict__ e, const V4<T>* m, T* uw,
                                            unsigned char* buf = nullptr) {
  T acc;
  if constexpr (PMFEM_COR_VW == 8 && PIPE > 0)
    acc = sell_dot8_pipe<PIPE>(cval, dcol, q + c0, cbase[t], coff[t >> 5] + 8 * (t & 31), clen[t], nc, buf);
  else if constexpr (PMFEM_COR_VW == 8)
    acc = sell_dot8<(PMFEM_COR_G + 1) / 2>(cval, dcol, q + c0, cbase[t], coff[t >> 5] + 8 * (t & 31), clen[t], nc);
  else
    acc = sell_dot4<PMFEM_COR_G>(cval, dcol, q + c0, cbase[t], coff[t >> 5] + 4 * (t & 31), clen[t], nc);
  acc += extras_row<T>(i, rowptrX, colX, valX, m);
  atomicAdd(uw + 4 * i, acc + e[i]);
}

// The two halves add into lane 3 of m, which enters every evaluation at zero (the permutation
// into the internal order and the RK stage updates write it so): the stencil pass can then run
// as soon as the FFT is done, while the precorrection may still run on the other stream, and the
// sum of the two adds is the same in either order (0 + a + b = 0 + b + a exactly).
template <typename T, int P>
__device__ __forceinline__ void stencil_add_row(int64_t i, const int32_t* __restrict__ base, const T* __restrict__ frac,
                                                const T* __restrict__ U, int N0, int N1, int N2, bool p0, bool p1,
                                                bool p2, T* uw) {
  atomicAdd(uw + 4 * i, stencil_row<T, P>(i, base, frac, U, N0, N1, N2, p0, p1, p2));
}

// ---------------------------------------------------------------- gradient + exchange + RK4
// Field of node i: gradient (Eq. 14d) and exchange (Eq. 8) over adjacency row i (vector
// width 4, as in charges_row; the potential u of a node is the fourth lane of its m vector),
// plus the applied field; then either the output (MODE 0, written to H[3 * uo] in the caller's
// order) or the RK4 stage update of the LLG equation (Eq. 2; MODE 1 an intermediate stage,
// MODE 2 the final combination with the renormalisation of Eq. 6 in FP64).
// Both operators annihilate constants (rows of the gradient and of the Laplacian sum to
// zero), so they act on differences to the row's own value: the same result in exact
// arithmetic, without the cancellation of large terms in floating point.
template <typename T, int MODE, typename CT, typename VG, typename VK, bool LOC = false>
__device__ __forceinline__ void field_row(int64_t i, int64_t c0, int32_t nc, const int32_t* __restrict__ len,
                                          const int32_t* __restrict__ base, const int64_t* __restrict__ off,
                                          const CT* __restrict__ dcol, const VG* __restrict__ gx,
                                          const VG* __restrict__ gy, const VG* __restrict__ gz,
                                          const VK* __restrict__ kp, const V4<T>* __restrict__ m, int64_t uo,
                                          T* __restrict__ H, int use_ms,
                                          int use_ex, T hx, T hy, T hz, V4<T>* __restrict__ m0,
                                          V4<T>* __restrict__ mnext, V4<T>* __restrict__ accb, T cdt, T bw,
                                          int acc_init, T dt6, T gam, T alpha, int* flag,
                                          LocalTerms<T> lt = LocalTerms<T>()) {
  const int ng = (len[i] + 3) >> 2;
  const int32_t b = base[i];
  int64_t o = off[i >> 5] + 4 * (i & 31);
  const V4<T> mn = m[i];           // (m, u) of node i: the potential sits in the fourth lane
  const T un = use_ms ? mn.w : T(0);
  const V4<T>* mc = m + c0;
  T ax = 0, ay = 0, az = 0;
  if (use_ms && use_ex) {
    for (int g = 0; g < ng; ++g, o += 128) {
      int32_t c[4];
      T g0[4], g1[4], g2[4], kk[4];
      ldc4(dcol + o, c);
      ldv4(gx + o, g0);
      ldv4(gy + o, g1);
      ldv4(gz + o, g2);
      ldv4(kp + o, kk);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const V4<T> mk = mc[col_of(b, c[k], nc)];   // one 16-byte gather: m and u of the neighbour
        const T du = mk.w - un;
        ax += g0[k] * du + kk[k] * (mk.x - mn.x);
        ay += g1[k] * du + kk[k] * (mk.y - mn.y);
        az += g2[k] * du + kk[k] * (mk.z - mn.z);
      }
    }
  } else if (use_ms) {
    for (int g = 0; g < ng; ++g, o += 128) {
      int32_t c[4];
      T g0[4], g1[4], g2[4];
      ldc4(dcol + o, c);
      ldv4(gx + o, g0);
      ldv4(gy + o, g1);
      ldv4(gz + o, g2);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T du = mc[col_of(b, c[k], nc)].w - un;
        ax += g0[k] * du;
        ay += g1[k] * du;
        az += g2[k] * du;
      }
    }
  } else if (use_ex) {
    for (int g = 0; g < ng; ++g, o += 128) {
      int32_t c[4];
      T kk[4];
      ldc4(dcol + o, c);
      ldv4(kp + o, kk);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const V4<T> mk = mc[col_of(b, c[k], nc)];
        ax += kk[k] * (mk.x - mn.x);
        ay += kk[k] * (mk.y - mn.y);
        az += kk[k] * (mk.z - mn.z);
      }
    }
  }
  if constexpr (LOC) {
    // anisotropy of the grains meeting at the node, weighted by their volume shares:
    // cubic -(2 K1/(mu0 Ms)) sum_i a_i (a_j^2 + a_k^2) axis_i, uniaxial (2 Ku/(mu0 Ms)) (m.u) u
    for (int32_t q = lt.ptr[i]; q < lt.ptr[i + 1]; ++q) {
      const T* P = lt.tab + kGrainTab * lt.grain[q];
      const T wq = lt.w[q];
      const T a1 = mn.x * P[0] + mn.y * P[1] + mn.z * P[2];
      const T a2 = mn.x * P[3] + mn.y * P[4] + mn.z * P[5];
      const T a3 = mn.x * P[6] + mn.y * P[7] + mn.z * P[8];
      const T s1 = a1 * a1, s2 = a2 * a2, s3 = a3 * a3;
      const T f1 = P[9] * a1 * (s2 + s3), f2 = P[9] * a2 * (s1 + s3), f3 = P[9] * a3 * (s1 + s2);
      const T mu = P[13] * (mn.x * P[10] + mn.y * P[11] + mn.z * P[12]);
      ax += wq * (f1 * P[0] + f2 * P[3] + f3 * P[6] + mu * P[10]);
      ay += wq * (f1 * P[1] + f2 * P[4] + f3 * P[7] + mu * P[11]);
      az += wq * (f1 * P[2] + f2 * P[5] + f3 * P[8] + mu * P[12]);
    }
  }
  const T Hx = ax + hx, Hy = ay + hy, Hz = az + hz;
  if (!(isfinite(Hx) && isfinite(Hy) && isfinite(Hz))) atomicOr(flag, FLAG_NONFINITE_OUT);
  if (MODE == 0) {
    H[3 * uo] = Hx;
    H[3 * uo + 1] = Hy;
    H[3 * uo + 2] = Hz;
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

}  // namespace
}  // namespace pmfem
