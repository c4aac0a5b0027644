// Learned surrogate of the FFT convolution (BAIM step 2): a 3D convolutional network on the
// AIM grid that maps grid charges Q to grid potential U.  Four 3x3x3 convolution layers
// (1 -> 32 -> 32 -> 32 -> 1 channels), the leaky rectifier act(z) = max(z, 0.1 z) after the
// first three, circular padding along periodic axes and zero padding along the others,
// fixed input and output scales sq and su.  Forward, backward (input and weight gradients)
// and the Adam update are hand-written kernels; weights, gradients and accumulation are FP32,
// hidden activations are stored in FP32 or (by choice) bfloat16.
//
// Layouts: a field of C channels is C planes of Z x Y x X floats (x fastest).  Weights are
// kept as W[tap][ci][co] (co fastest) so that the forward kernel reads one contiguous row of
// output-channel weights per (tap, input channel); the caller's parameter order is the usual
// W[co][ci][dz][dy][dx] followed by b[co], layer after layer.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pmfem.h"
#include "device.hpp"
#include "internal.hpp"
#include "surrogate.hpp"

namespace pmfem {
namespace {

constexpr int TX = 8, TY = 8, TZ = 4;                // output tile of one block
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;  // with its halo
constexpr int HALO = HX * HY * HZ;                    // 600
constexpr int TILE = TX * TY * TZ;                    // 256 threads, one voxel each
constexpr float kSlope = 0.1f;

template <typename A> __device__ __forceinline__ float ld_act(const A* p);
template <> __device__ __forceinline__ float ld_act<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_act<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <typename A> __device__ __forceinline__ void st_act(A* p, float v);
template <> __device__ __forceinline__ void st_act<float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st_act<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ int wrapc(int i, int n, bool per, bool& inside) {
  inside = true;
  if (i < 0) {
    if (per) return i + n;
    inside = false;
  } else if (i >= n) {
    if (per) return i - n;
    inside = false;
  }
  return i;
}

// Halo tile of CK input channels starting at c0 into s[CK][HALO], scaled by scale; padding per axis.
template <int CK, typename AIN, bool CL = false>
__device__ __forceinline__ void load_halo(float* s, const AIN* __restrict__ in, int c0, int Cin, int X, int Y, int Z,
                                          int x0, int y0, int z0, bool px, bool py, bool pz, float scale) {
  const int64_t plane = (int64_t)X * Y * Z;
  for (int k = threadIdx.x; k < CK * HALO; k += blockDim.x) {
    const int c = k / HALO, h = k - c * HALO;
    const int hz = h / (HX * HY), hy = (h / HX) % HY, hx = h % HX;
    bool ix, iy, iz;
    const int gx = wrapc(x0 + hx - 1, X, px, ix), gy = wrapc(y0 + hy - 1, Y, py, iy), gz = wrapc(z0 + hz - 1, Z, pz, iz);
    float v = 0.f;
    const int64_t vox = gx + (int64_t)X * (gy + (int64_t)Y * gz);
    if (c0 + c < Cin && ix && iy && iz) v = scale * ld_act(in + (CL ? vox * Cin + c0 + c : (int64_t)(c0 + c) * plane + vox));
    s[k] = v;
  }
}

// y[co] = act?(b[co] + sum_ci sum_tap W[tap][ci][co] x[ci](v + tap - 1)) * oscale for a tile.
// Cin arbitrary (chunks of CK), COUT <= 32 output channels, one voxel per thread.
template <int CK, int COUT, bool ACT, typename AIN, typename AOUT, bool CL_IN = false, bool CL_OUT = false>
__global__ void __launch_bounds__(TILE) k_conv_fwd(const AIN* __restrict__ in, int Cin, const float* __restrict__ W,
                                                   const float* __restrict__ b, AOUT* __restrict__ out, int X, int Y,
                                                   int Z, bool px, bool py, bool pz, float in_scale, float out_scale,
                                                   AOUT* __restrict__ pout = nullptr) {
  __shared__ float s_in[CK * HALO];
  __shared__ __align__(16) float s_w[27 * CK * COUT];
  const int ntx = X / TX, nty = Y / TY;
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * TX, y0 = ((tile / ntx) % nty) * TY, z0 = (tile / (ntx * nty)) * TZ;
  const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = b ? b[o] : 0.f;
  for (int c0 = 0; c0 < Cin; c0 += CK) {
    __syncthreads();
    load_halo<CK, AIN, CL_IN>(s_in, in, c0, Cin, X, Y, Z, x0, y0, z0, px, py, pz, in_scale);
    for (int k = threadIdx.x; k < 27 * CK * COUT; k += blockDim.x) {
      const int tap = k / (CK * COUT), r = k - tap * CK * COUT, ci = r / COUT;
      s_w[k] = (c0 + ci < Cin) ? W[((int64_t)tap * Cin + c0 + ci) * COUT + (r - ci * COUT)] : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int tap = 0; tap < 27; ++tap) {
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      const int h = (lz + dz) * HX * HY + (ly + dy) * HX + lx + dx;
#pragma unroll
      for (int ci = 0; ci < CK; ++ci) {
        const float v = s_in[ci * HALO + h];
        const float* w = s_w + (tap * CK + ci) * COUT;
        if constexpr (COUT % 4 == 0) {   // one 16-byte (broadcast) weight load per 4 FMAs
#pragma unroll
          for (int o = 0; o < COUT; o += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(w + o);
            acc[o] += v * w4.x, acc[o + 1] += v * w4.y, acc[o + 2] += v * w4.z, acc[o + 3] += v * w4.w;
          }
        } else {
#pragma unroll
          for (int o = 0; o < COUT; ++o) acc[o] += v * w[o];
        }
      }
    }
  }
  const int64_t plane = (int64_t)X * Y * Z;
  const int64_t vox = (x0 + lx) + (int64_t)X * ((y0 + ly) + (int64_t)Y * (z0 + lz));
  if constexpr (CL_OUT && sizeof(AOUT) == 2 && COUT % 8 == 0) {   // channels-last bfloat16: 16-byte stores
    // (and, when pout is set, the same rows in the padded layout the tensor-core layer reads)
    int64_t slot[8];
    const int ns = pout ? pad_slots(x0 + lx, y0 + ly, z0 + lz, X, Y, Z, px, py, pz, slot) : 0;
    const int64_t vp = (int64_t)(X + 2) * (Y + 2) * (Z + 2);   // voxels of one padded group plane
#pragma unroll
    for (int o = 0; o < COUT; o += 8) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float a = acc[o + 2 * j], c = acc[o + 2 * j + 1];
        if (ACT) a = a > 0.f ? a : kSlope * a, c = c > 0.f ? c : kSlope * c;
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(a * out_scale, c * out_scale);
        w[j] = *reinterpret_cast<const uint32_t*>(&p2);
      }
      const uint4 v = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(out + vox * COUT + o) = v;
      for (int k = 0; k < ns; ++k) *reinterpret_cast<uint4*>(pout + ((o / 8) * vp + slot[k]) * 8) = v;
    }
  } else {
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      float z = acc[o];
      if (ACT) z = z > 0.f ? z : kSlope * z;
      st_act(out + (CL_OUT ? vox * COUT + o : (int64_t)o * plane + vox), z * out_scale);
    }
  }
}

// Output layer (32 -> 1, no activation) on channels-last bfloat16 activations: the block's
// halo with all 32 channels (600 voxels x 64 B) is staged with 16-byte loads, then each
// thread sums 27 taps x 32 channels for its voxel.  W is [tap][ci] (one output channel).
// Piece g of halo voxel h sits at 4 h + (g ^ ((h >> 1) & 3)): eight consecutive voxels then
// fall in eight different 16-byte bank groups (unswizzled, the 64-byte voxel stride makes
// the eight lanes of a phase collide four ways).
__global__ void __launch_bounds__(TILE) k_conv_out_cl(const __nv_bfloat16* __restrict__ in, const float* __restrict__ W,
                                                      const float* __restrict__ b, float* __restrict__ out, int X,
                                                      int Y, int Z, bool px, bool py, bool pz, float out_scale) {
  __shared__ uint4 s_in[HALO * 4];
  __shared__ float4 s_w4[27 * 8];
  float* s_w = reinterpret_cast<float*>(s_w4);
  const int ntx = X / TX, nty = Y / TY;
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * TX, y0 = ((tile / ntx) % nty) * TY, z0 = (tile / (ntx * nty)) * TZ;
  for (int k = threadIdx.x; k < 27 * 32; k += blockDim.x) s_w[k] = W[k];
  // every 16-byte piece is one cp.async, all in flight at once (zero fill outside a
  // non-periodic border: source size 0, nothing read)
  for (int k = threadIdx.x; k < HALO * 4; k += blockDim.x) {
    const int h = k >> 2, g = k & 3;
    const int hz = h / (HX * HY), hy = (h / HX) % HY, hx = h % HX;
    bool ix, iy, iz;
    const int gx = wrapc(x0 + hx - 1, X, px, ix), gy = wrapc(y0 + hy - 1, Y, py, iy), gz = wrapc(z0 + hz - 1, Z, pz, iz);
    const bool inside = ix && iy && iz;
    const uint4* src = reinterpret_cast<const uint4*>(in) +
                       (inside ? 4 * (gx + (int64_t)X * (gy + (int64_t)Y * gz)) + g : 0);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_in + 4 * h + (g ^ ((h >> 1) & 3)));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(inside ? 16u : 0u)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
  float acc = b[0];
#pragma unroll 1
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int h = (lz + dz) * HX * HY + (ly + dy) * HX + lx + dx;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const uint4 v = s_in[4 * h + (g ^ ((h >> 1) & 3))];
      const float4 wa = s_w4[8 * tap + 2 * g], wb = s_w4[8 * tap + 2 * g + 1];   // channels 8g .. 8g+7
      acc += wa.x * __uint_as_float(v.x << 16) + wa.y * __uint_as_float(v.x & 0xffff0000u);
      acc += wa.z * __uint_as_float(v.y << 16) + wa.w * __uint_as_float(v.y & 0xffff0000u);
      acc += wb.x * __uint_as_float(v.z << 16) + wb.y * __uint_as_float(v.z & 0xffff0000u);
      acc += wb.z * __uint_as_float(v.w << 16) + wb.w * __uint_as_float(v.w & 0xffff0000u);
    }
  }
  out[(x0 + lx) + (int64_t)X * ((y0 + ly) + (int64_t)Y * (z0 + lz))] = acc * out_scale;
}

// g[c](v) *= act'(h[c](v)), read from the activation h (act keeps the sign of its argument).
template <typename A, bool CL = false>
__global__ void k_act_bwd(float* __restrict__ g, const A* __restrict__ h, int64_t n, int64_t V, int C) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // g is planar: i = c V + v
  if (i >= n) return;
  const int64_t hi = CL ? (i % V) * C + i / V : i;
  if (!(ld_act(h + hi) > 0.f)) g[i] *= kSlope;
}

// Weights of the input-gradient convolution: the adjoint of y = W * x is x' = W' * y with
// W'[tap][co][ci] = W[26 - tap][ci][co] (the kernel mirrored, channels swapped).
__global__ void k_flip(const float* __restrict__ W, float* __restrict__ Wt, int Cin, int Cout) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 27 * Cin * Cout) return;
  const int tap = k / (Cin * Cout), r = k - tap * Cin * Cout, ci = r / Cout, co = r - ci * Cout;
  Wt[((int64_t)(26 - tap) * Cout + co) * Cin + ci] = W[k];
}

// dW[tap][ci][co] += sum_v g[co](v) x[ci](v + tap - 1) and db[co] += sum_v g[co](v), over
// the tiles of this block (grid-stride), one (ci, co) pair per thread with 27 accumulators.
template <int CI, int CO, typename AIN, bool CL_IN = false>
__global__ void __launch_bounds__(1024) k_conv_wgrad(const AIN* __restrict__ x, const float* __restrict__ g, int X,
                                                    int Y, int Z, bool px, bool py, bool pz, float in_scale,
                                                    float* __restrict__ dW, float* __restrict__ db) {
  extern __shared__ float smem[];
  float* s_x = smem;                // CI x HALO
  float* s_g = smem + CI * HALO;    // CO x TILE
  const int ntx = X / TX, nty = Y / TY, ntiles = ntx * nty * (Z / TZ);
  const int pair = threadIdx.x, ci = pair / CO, co = pair % CO;
  const bool active = pair < CI * CO;
  float acc[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) acc[t] = 0.f;
  float accb = 0.f;
  const int64_t plane = (int64_t)X * Y * Z;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x0 = (tile % ntx) * TX, y0 = ((tile / ntx) % nty) * TY, z0 = (tile / (ntx * nty)) * TZ;
    __syncthreads();
    load_halo<CI, AIN, CL_IN>(s_x, x, 0, CI, X, Y, Z, x0, y0, z0, px, py, pz, in_scale);
    for (int k = threadIdx.x; k < CO * TILE; k += blockDim.x) {
      const int c = k / TILE, v = k - c * TILE;
      const int lx = v % TX, ly = (v / TX) % TY, lz = v / (TX * TY);
      s_g[k] = g[(int64_t)c * plane + (x0 + lx) + (int64_t)X * ((y0 + ly) + (int64_t)Y * (z0 + lz))];
    }
    __syncthreads();
    if (active) {
#pragma unroll 1
      for (int v = 0; v < TILE; ++v) {
        const int lx = v % TX, ly = (v / TX) % TY, lz = v / (TX * TY);
        const float gv = s_g[co * TILE + v];
        const float* xs = s_x + ci * HALO + lz * HX * HY + ly * HX + lx;
        accb += gv;
#pragma unroll
        for (int t = 0; t < 27; ++t) acc[t] += gv * xs[(t / 9) * HX * HY + ((t / 3) % 3) * HX + t % 3];
      }
    }
  }
  if (active) {
#pragma unroll
    for (int t = 0; t < 27; ++t) atomicAdd(&dW[((int64_t)t * CI + ci) * CO + co], acc[t]);
    if (ci == 0) atomicAdd(&db[co], accb);
  }
}

// r = (pred - U) / su; g = 2 r / n (gradient of the mean squared error in units of su with
// respect to the last layer's output, which is pred / su); loss += sum r^2 / n.
__global__ void k_out_grad(const float* __restrict__ pred, const float* __restrict__ U, float* __restrict__ g,
                           int64_t n, float inv_su, double* __restrict__ loss) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float r2 = 0.f;
  if (i < n) {
    const float r = (pred[i] - U[i]) * inv_su;
    g[i] = 2.f * r / (float)n;
    r2 = r * r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0 && r2 != 0.f) atomicAdd(loss, (double)r2 / (double)n);
}

// Adam (Kingma and Ba, 2015) on n parameters; bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ a, const float* __restrict__ b, float s,
                       int64_t n) {   // y = a + s * b
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] + s * b[i];
}

inline unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace
}  // namespace pmfem

namespace pmfem {
namespace {

__global__ void k_err_acc(const float* __restrict__ a, const float* __restrict__ ref, int64_t n, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.f, r2 = 0.f;
  if (i < n) {
    const float d = a[i] - ref[i];
    d2 = d * d;
    r2 = ref[i] * ref[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, (double)d2);
    atomicAdd(out + 1, (double)r2);
  }
}

template <typename K>
void opt_in_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

unsigned ntiles(const SurrogateNet& n) { return (unsigned)((n.dims[0] / TX) * (n.dims[1] / TY) * (n.dims[2] / TZ)); }

template <int CI, int CO, typename A, bool CL = false>
void wgrad(const SurrogateNet& n, const A* x, const float* g, float in_scale, int layer, cudaStream_t st) {
  const size_t sm = (size_t)(CI * HALO + CO * TILE) * sizeof(float);
  opt_in_smem(k_conv_wgrad<CI, CO, A, CL>, sm);
  const unsigned nb = std::min(ntiles(n), 2u * 152u);
  k_conv_wgrad<CI, CO, A, CL><<<nb, 1024, sm, st>>>(x, g, n.dims[0], n.dims[1], n.dims[2], n.periodic[0], n.periodic[1],
                                               n.periodic[2], in_scale, n.G + net_layer_offset(layer, false),
                                               n.G + net_layer_offset(layer, true));
}

template <typename A>
void forward_t(SurrogateNet& n, const float* Q, float* U, cudaStream_t st) {
  const unsigned nt = ntiles(n);
  const int X = n.dims[0], Y = n.dims[1], Z = n.dims[2];
  const bool px = n.periodic[0], py = n.periodic[1], pz = n.periodic[2];
  A* h0 = (A*)n.h[0];
  A* h1 = (A*)n.h[1];
  A* h2 = (A*)n.h[2];
  if constexpr (sizeof(A) == 2) {
    if (n.tc) {   // channels-last activations, layers 1 and 2 on the tensor cores
      conv32_tc_pack(n.W[1], n.Wp[0], st);
      conv32_tc_pack(n.W[2], n.Wp[1], st);
      n.prof.begin(KID_SUR_IN, st);
      k_conv_fwd<1, kNetC, true, float, A, false, true><<<nt, TILE, 0, st>>>(Q, 1, n.W[0], n.b[0], h0, X, Y, Z, px, py,
                                                                              pz, 1.f / n.sq, 1.f, (A*)n.hpad[0]);
      n.prof.end(KID_SUR_IN, st);
      n.prof.begin(KID_SUR_HIDDEN, st);
      conv32_tc(n.tmap[0], n.Wp[0], n.b[1], h1, n.hpad[1], n.dims, n.periodic, true, n.tc_err, st);
      n.prof.end(KID_SUR_HIDDEN, st);
      n.prof.begin(KID_SUR_HIDDEN, st);
      conv32_tc(n.tmap[1], n.Wp[1], n.b[2], h2, nullptr, n.dims, n.periodic, true, n.tc_err, st);
      n.prof.end(KID_SUR_HIDDEN, st);
      n.prof.begin(KID_SUR_OUT, st);
      k_conv_out_cl<<<nt, TILE, 0, st>>>(h2, n.W[3], n.b[3], U, X, Y, Z, px, py, pz, n.su);
      n.prof.end(KID_SUR_OUT, st);
      return;
    }
  }
  n.prof.begin(KID_SUR_IN, st);
  k_conv_fwd<1, kNetC, true, float, A><<<nt, TILE, 0, st>>>(Q, 1, n.W[0], n.b[0], h0, X, Y, Z, px, py, pz, 1.f / n.sq, 1.f);
  n.prof.end(KID_SUR_IN, st);
  n.prof.begin(KID_SUR_HIDDEN, st);
  k_conv_fwd<8, kNetC, true, A, A><<<nt, TILE, 0, st>>>(h0, kNetC, n.W[1], n.b[1], h1, X, Y, Z, px, py, pz, 1.f, 1.f);
  n.prof.end(KID_SUR_HIDDEN, st);
  n.prof.begin(KID_SUR_HIDDEN, st);
  k_conv_fwd<8, kNetC, true, A, A><<<nt, TILE, 0, st>>>(h1, kNetC, n.W[2], n.b[2], h2, X, Y, Z, px, py, pz, 1.f, 1.f);
  n.prof.end(KID_SUR_HIDDEN, st);
  n.prof.begin(KID_SUR_OUT, st);
  k_conv_fwd<8, 1, false, A, float><<<nt, TILE, 0, st>>>(h2, kNetC, n.W[3], n.b[3], U, X, Y, Z, px, py, pz, 1.f, n.su);
  n.prof.end(KID_SUR_OUT, st);
}

// Backward pass: the input gradients run as convolutions with mirrored weights (planar FP32
// gradient buffers, CUDA cores); CL says whether the stored activations are channels-last.
template <typename A, bool CL>
void backward_layers(SurrogateNet& n, const float* Q, cudaStream_t st) {
  const unsigned nt = ntiles(n);
  const int X = n.dims[0], Y = n.dims[1], Z = n.dims[2];
  const bool px = n.periodic[0], py = n.periodic[1], pz = n.periodic[2];
  const int64_t V = n.V, VC = (int64_t)kNetC * V;
  const A* h0 = (const A*)n.h[0];
  const A* h1 = (const A*)n.h[1];
  const A* h2 = (const A*)n.h[2];
  // layer 3: 32 -> 1
  wgrad<kNetC, 1, A, CL>(n, h2, n.gA, 1.f, 3, st);
  k_flip<<<nb256(27 * kNetC), 256, 0, st>>>(n.W[3], n.Wt, kNetC, 1);
  k_conv_fwd<1, kNetC, false, float, float><<<nt, TILE, 0, st>>>(n.gA, 1, n.Wt, nullptr, n.gB, X, Y, Z, px, py, pz, 1.f, 1.f);
  k_act_bwd<A, CL><<<nb256(VC), 256, 0, st>>>(n.gB, h2, VC, V, kNetC);
  // layer 2: 32 -> 32
  wgrad<kNetC, kNetC, A, CL>(n, h1, n.gB, 1.f, 2, st);
  k_flip<<<nb256(27 * kNetC * kNetC), 256, 0, st>>>(n.W[2], n.Wt, kNetC, kNetC);
  k_conv_fwd<8, kNetC, false, float, float><<<nt, TILE, 0, st>>>(n.gB, kNetC, n.Wt, nullptr, n.gA, X, Y, Z, px, py, pz, 1.f, 1.f);
  k_act_bwd<A, CL><<<nb256(VC), 256, 0, st>>>(n.gA, h1, VC, V, kNetC);
  // layer 1: 32 -> 32
  wgrad<kNetC, kNetC, A, CL>(n, h0, n.gA, 1.f, 1, st);
  k_flip<<<nb256(27 * kNetC * kNetC), 256, 0, st>>>(n.W[1], n.Wt, kNetC, kNetC);
  k_conv_fwd<8, kNetC, false, float, float><<<nt, TILE, 0, st>>>(n.gA, kNetC, n.Wt, nullptr, n.gB, X, Y, Z, px, py, pz, 1.f, 1.f);
  k_act_bwd<A, CL><<<nb256(VC), 256, 0, st>>>(n.gB, h0, VC, V, kNetC);
  // layer 0: 1 -> 32, input Q / sq
  wgrad<1, kNetC, float, false>(n, Q, n.gB, 1.f / n.sq, 0, st);
}

template <typename A>
void backward_t(SurrogateNet& n, const float* Q, const float* Ut, cudaStream_t st) {
  forward_t<A>(n, Q, n.pred, st);
  k_out_grad<<<nb256(n.V), 256, 0, st>>>(n.pred, Ut, n.gA, n.V, 1.f / n.su, n.loss);
  if (sizeof(A) == 2 && n.tc)
    backward_layers<A, true>(n, Q, st);
  else
    backward_layers<A, false>(n, Q, st);
}

}  // namespace

int64_t net_layer_offset(int layer, bool bias) {
  static const int ci[4] = {1, kNetC, kNetC, kNetC}, co[4] = {kNetC, kNetC, kNetC, 1};
  int64_t o = 0;
  for (int k = 0; k < layer; ++k) o += 27 * ci[k] * co[k] + co[k];
  return bias ? o + 27 * ci[layer] * co[layer] : o;
}

void net_params_to_device_layout(const float* in, std::vector<float>& out) {
  static const int ci[4] = {1, kNetC, kNetC, kNetC}, co[4] = {kNetC, kNetC, kNetC, 1};
  out.assign(kNetParams, 0.f);
  for (int k = 0; k < 4; ++k) {
    const int64_t o = net_layer_offset(k, false);
    for (int c = 0; c < co[k]; ++c)
      for (int i = 0; i < ci[k]; ++i)
        for (int t = 0; t < 27; ++t) out[o + ((int64_t)t * ci[k] + i) * co[k] + c] = in[o + ((int64_t)c * ci[k] + i) * 27 + t];
    const int64_t ob = net_layer_offset(k, true);
    for (int c = 0; c < co[k]; ++c) out[ob + c] = in[ob + c];
  }
}

void net_params_from_device_layout(const float* in, std::vector<float>& out) {
  static const int ci[4] = {1, kNetC, kNetC, kNetC}, co[4] = {kNetC, kNetC, kNetC, 1};
  out.assign(kNetParams, 0.f);
  for (int k = 0; k < 4; ++k) {
    const int64_t o = net_layer_offset(k, false);
    for (int c = 0; c < co[k]; ++c)
      for (int i = 0; i < ci[k]; ++i)
        for (int t = 0; t < 27; ++t) out[o + ((int64_t)c * ci[k] + i) * 27 + t] = in[o + ((int64_t)t * ci[k] + i) * co[k] + c];
    const int64_t ob = net_layer_offset(k, true);
    for (int c = 0; c < co[k]; ++c) out[ob + c] = in[ob + c];
  }
}

int net_create(SurrogateNet& n, const int dims[3], const bool periodic[3], bool bf16, std::string& msg) {
  if (dims[0] % TX || dims[1] % TY || dims[2] % TZ) {
    msg = "the surrogate needs grid dimensions that are multiples of 8, 8 and 4";
    return EINVAL_;
  }
  for (int a = 0; a < 3; ++a) n.dims[a] = dims[a], n.periodic[a] = periodic[a];
  n.bf16 = bf16;
  n.V = (int64_t)dims[0] * dims[1] * dims[2];
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    n.allocs.push_back(*p);
    return cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  void* p;
  const size_t pb = kNetParams * sizeof(float);
  bool ok = alloc(&p, pb) && ((n.P = (float*)p), true) && alloc(&p, pb) && ((n.G = (float*)p), true) &&
            alloc(&p, pb) && ((n.M = (float*)p), true) && alloc(&p, pb) && ((n.S2 = (float*)p), true) &&
            alloc(&p, 27 * kNetC * kNetC * sizeof(float)) && ((n.Wt = (float*)p), true);
  const size_t ab = (size_t)kNetC * n.V * (bf16 ? 2 : 4);
  for (int k = 0; k < 3 && ok; ++k) ok = alloc(&n.h[k], ab);
  ok = ok && alloc(&p, (size_t)kNetC * n.V * 4) && ((n.gA = (float*)p), true) &&
       alloc(&p, (size_t)kNetC * n.V * 4) && ((n.gB = (float*)p), true) && alloc(&p, n.V * 4) &&
       ((n.pred = (float*)p), true) && alloc(&p, n.V * 4) && ((n.Q1 = (float*)p), true) && alloc(&p, n.V * 4) &&
       ((n.U1 = (float*)p), true) && alloc(&p, n.V * 4) && ((n.Ubuf = (float*)p), true) &&
       alloc(&p, 2 * sizeof(double)) && ((n.loss = (double*)p), true) && alloc(&p, 2 * sizeof(double)) &&
       ((n.err = (double*)p), true);
  n.tc = bf16 && conv32_tc_fits(dims);
  const size_t padb = (size_t)kNetC * 2 * (dims[0] + 2) * (dims[1] + 2) * (dims[2] + 2);
  if (ok && n.tc)
    ok = alloc(&n.Wp[0], 27 * kNetC * kNetC * 2) && alloc(&n.Wp[1], 27 * kNetC * kNetC * 2) &&
         alloc(&p, sizeof(int)) && ((n.tc_err = (int*)p), true) && alloc(&n.hpad[0], padb) &&
         alloc(&n.hpad[1], padb);
  if (!ok) {
    net_destroy(n);
    msg = "device allocation for the surrogate failed";
    return ENOMEM_;
  }
  if (n.tc && !(conv32_tc_tensor_map(n.hpad[0], dims, n.tmap[0]) && conv32_tc_tensor_map(n.hpad[1], dims, n.tmap[1]))) {
    net_destroy(n);
    msg = "tensor map of the surrogate's padded activations could not be encoded";
    return ECUDA_;
  }
  for (int k = 0; k < 4; ++k) n.W[k] = n.P + net_layer_offset(k, false), n.b[k] = n.P + net_layer_offset(k, true);
  return OK;
}

void net_destroy(SurrogateNet& n) {
  for (void* p : n.allocs) cudaFree(p);
  n = SurrogateNet();
}

void net_forward(SurrogateNet& n, const float* Q, float* U, cudaStream_t st) {
  if (n.bf16)
    forward_t<__nv_bfloat16>(n, Q, U, st);
  else
    forward_t<float>(n, Q, U, st);
}

void net_backward(SurrogateNet& n, const float* Q, const float* U, cudaStream_t st) {
  if (n.bf16)
    backward_t<__nv_bfloat16>(n, Q, U, st);
  else
    backward_t<float>(n, Q, U, st);
}

void net_adam(SurrogateNet& n, float lr, int64_t t, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<nb256(kNetParams), 256, 0, st>>>(n.P, n.G, n.M, n.S2, kNetParams, lr, b1, b2, 1e-8f,
                                            (float)(1.0 - std::pow(0.9, (double)t)),
                                            (float)(1.0 - std::pow(0.999, (double)t)));
}

void net_increment(SurrogateNet& n, float* grid, cudaStream_t st) {
  k_axpy<<<nb256(n.V), 256, 0, st>>>(n.pred, grid, n.Q1, -1.f, n.V);   // dQ = Q - Q1
  net_forward(n, n.pred, n.Ubuf, st);
  k_axpy<<<nb256(n.V), 256, 0, st>>>(grid, n.U1, n.Ubuf, 1.f, n.V);    // U = U1 + net(dQ)
}

void net_judge(SurrogateNet& n, const float* Qs, const float* U, cudaStream_t st) {
  k_axpy<<<nb256(n.V), 256, 0, st>>>(n.pred, Qs, n.Q1, -1.f, n.V);
  net_forward(n, n.pred, n.Ubuf, st);
  k_axpy<<<nb256(n.V), 256, 0, st>>>(n.Ubuf, n.U1, n.Ubuf, 1.f, n.V);
  k_err_acc<<<nb256(n.V), 256, 0, st>>>(n.Ubuf, U, n.V, n.err);
}

}  // namespace pmfem
