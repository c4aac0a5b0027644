// 32 -> 32 channel 3x3x3 convolution of the surrogate network on the 5th-generation tensor
// cores (tcgen05): an implicit GEMM D[128 voxels][32 out] = sum over 27 taps of
// A_tap[128 voxels][32 in] * W_tap[32 out][32 in]^T, BF16 operands in shared memory, FP32
// accumulator in tensor memory.
//
// A tile is 8 (x) x 16 (y) x 1 (z) output voxels (M = 128); one persistent block per SM walks
// the tiles.  For each tile the block stages the
// input halo (10 x 18 x 3 voxels) in shared memory as four planes of 8 channels, so that the
// 8 channels of one voxel are one 16-byte row: for tap (dx, dy, dz) the A operand of an MMA is
// the halo seen from offset (dx, dy, dz) -- 8 consecutive x voxels form one 8 x 16-byte core
// matrix, the 16 y rows of the tile sit 10 voxels apart (stride-dimension offset 160 B), and
// the next 8 channels sit one plane further (leading-dimension offset 540 x 16 B).  No im2col
// copy is made; each tap is two MMAs of K = 16 (channels 0-15 and 16-31).  The weights of all
// 27 taps are staged once as [tap][channel group][out][8 in] (K-major core matrices).
//
// Activations in global memory are channels-last BF16, [voxel][32].
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "device.hpp"
#include "surrogate.hpp"

namespace pmfem {
namespace {

constexpr int CX = 8, CY = 16;                       // output tile (x, y); one z plane
constexpr int HX = CX + 2, HY = CY + 2, HZ = 3;      // halo
constexpr int HVOX = HX * HY * HZ;                   // 540 voxels
constexpr int WELEMS = 27 * 4 * 32 * 8;              // packed weights, bf16 elements
constexpr int SMEM_W = WELEMS * 2;                   // 55296 B
constexpr int SMEM_X = 4 * HVOX * 16;                // 34560 B
// + mbarrier and TMEM address.  Every descriptor this kernel forms stays inside s_w and s_x:
// the largest A read is the tap offset ((2 HY + 2) HX + 2) x 16 B, plus the half-K offset
// 2 x 540 x 16 B, one more K core matrix (540 x 16 B), 15 row groups of 160 B and one core
// matrix of 128 B, which is exactly SMEM_X (one halo buffer); the largest B read ends exactly
// at SMEM_W.
// halo buffers of the persistent kernel: 1 (two blocks per SM, each overlapping the other) or
// 2 (one block per SM, the next halo copied during the MMAs); measured on a 64^3 grid: 1 buffer
// with the weights resident beats both 2 buffers and a non-persistent block per tile
#ifndef PMFEM_TC_NBUF
#define PMFEM_TC_NBUF 1
#endif
constexpr int SMEM_TOTAL = SMEM_W + PMFEM_TC_NBUF * SMEM_X + 128;   // weights, halo buffers, barrier
static_assert(((2 * HY + 2) * HX + 2) * 16 + 2 * HVOX * 16 + HVOX * 16 + 15 * HX * 16 + 128 == SMEM_X, "A extent");
static_assert(((26 * 4 + 2) * 32 + 32 + 3 * 8) * 16 + 128 == SMEM_W, "B extent");
constexpr int kWaitIters = 1 << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// (K direction) and stride-dimension (M/N direction) byte offsets between core matrices,
// all >> 4; bits 46-48 hold the descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitIters; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16-byte global -> shared copy; the bytes past src_bytes (all 16 when it is 0) are zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ int wrap_in(int i, int n, bool per, bool& inside) {
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

// W[tap][ci][co] (FP32) -> Wp[tap][ci / 8][co][ci % 8] (BF16)
__global__ void k_pack_w32(const float* __restrict__ W, __nv_bfloat16* __restrict__ Wp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 27 * 32 * 32) return;
  const int tap = k >> 10, r = k & 1023, ci = r >> 5, co = r & 31;
  Wp[((tap * 4 + (ci >> 3)) * 32 + co) * 8 + (ci & 7)] = __float2bfloat16_rn(W[k]);
}

// Halo of output tile `tile` into buffer s_x (four channel-group planes), one 16-byte cp.async
// per piece, zero fill outside non-periodic borders (source size 0: nothing is read).
__device__ __forceinline__ void stage_halo(uint4* s_x, const __nv_bfloat16* __restrict__ in, int tile, int X, int Y,
                                           int Z, bool px, bool py, bool pz) {
  const int ntx = X / CX, nty = Y / CY;
  const int x0 = (tile % ntx) * CX, y0 = ((tile / ntx) % nty) * CY, z0 = tile / (ntx * nty);
  for (int k = threadIdx.x; k < 4 * HVOX; k += blockDim.x) {
    const int h = k >> 2, cg = k & 3;
    const int hz = h / (HX * HY), hy = (h / HX) % HY, hx = h % HX;
    bool ix, iy, iz;
    const int gx = wrap_in(x0 + hx - 1, X, px, ix), gy = wrap_in(y0 + hy - 1, Y, py, iy);
    const int gz = wrap_in(z0 + hz - 1, Z, pz, iz);
    const bool inside = ix && iy && iz;
    const uint4* src = reinterpret_cast<const uint4*>(in) +
                       (inside ? 4 * (gx + (int64_t)X * (gy + (int64_t)Y * gz)) + cg : 0);
    cp_async16(smem_u32(s_x + cg * HVOX + h), src, inside ? 16 : 0);
  }
}

// Persistent form: each block walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... with the
// weights staged once.  NBUF = 2: one block per SM, the halo double-buffered, so the next
// tile's halo is copied while the current tile's MMAs run.  NBUF = 1: two blocks per SM, the
// next halo copied into the single buffer once the MMAs that read it have completed (during the
// epilogue); the other block of the SM fills the gaps.  One 32-column TMEM accumulator is
// drained by the epilogue before the next tile's MMAs are issued (the block barrier at the end
// of each iteration orders the two).  The commit barrier completes one phase per tile.
template <int NBUF>
__global__ void __launch_bounds__(128, 3 - NBUF) k_conv32_tc(const __nv_bfloat16* __restrict__ in,
                                                     const __nv_bfloat16* __restrict__ Wp,
                                                     const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                     int X, int Y, int Z, bool px, bool py, bool pz, int act,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint4* s_w = reinterpret_cast<uint4*>(smem);
  uint4* s_x = reinterpret_cast<uint4*>(smem + SMEM_W);   // buffer b at s_x + b * 4 * HVOX
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SMEM_W + NBUF * SMEM_X);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SMEM_W + NBUF * SMEM_X + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntx = X / CX, nty = Y / CY, ntiles = ntx * nty * Z;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const uint4* wg = reinterpret_cast<const uint4*>(Wp);
  for (int k = tid; k < SMEM_W / 16; k += blockDim.x) cp_async16(smem_u32(s_w + k), wg + k, 16);
  if ((int)blockIdx.x < ntiles) stage_halo(s_x, in, blockIdx.x, X, Y, Z, px, py, pz);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t ws = smem_u32(s_w);

  int it = 0;
  bool ok = true;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = NBUF == 2 ? (it & 1) : 0;
    if (tid == 0) {
      const uint32_t xs = smem_u32(s_x + b * 4 * HVOX);
      for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const uint32_t aoff = (uint32_t)(((dz * HY + dy) * HX + dx) * 16);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const uint64_t adesc = smem_desc(xs + aoff + (uint32_t)(half * 2 * HVOX * 16), HVOX * 16, HX * 16);
          const uint64_t bdesc = smem_desc(ws + (uint32_t)((tap * 4 + half * 2) * 32 * 16), 32 * 16, 8 * 16);
          const uint32_t accum = (tap | half) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                   : "memory");
    }
    // the next tile's halo goes to the other buffer while these MMAs run (that buffer's last
    // reader, the previous tile's MMAs, completed before the previous epilogue)
    const int next = tile + gridDim.x;
    if (NBUF == 2 && next < ntiles) stage_halo(s_x + (b ^ 1) * 4 * HVOX, in, next, X, Y, Z, px, py, pz);
    ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(bar), (uint32_t)(it & 1)));   // warp-uniform for tcgen05.ld
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // one buffer: the MMAs that read it have completed (commit observed), so the next halo can
    // be copied into it while the epilogue runs
    if (NBUF == 1 && ok && next < ntiles) stage_halo(s_x, in, next, X, Y, Z, px, py, pz);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (ok) {
      const int x0 = (tile % ntx) * CX, y0 = ((tile / ntx) % nty) * CY, z0 = tile / (ntx * nty);
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int m = tid;   // row = lane of TMEM = voxel (x0 + m % 8, y0 + m / 8, z0)
      const int64_t vox = (x0 + (m & 7)) + (int64_t)X * ((y0 + (m >> 3)) + (int64_t)Y * z0);
      uint32_t packed[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float a = __uint_as_float(r[2 * c]) + bias[2 * c];
        float bb = __uint_as_float(r[2 * c + 1]) + bias[2 * c + 1];
        if (act) {
          a = a > 0.f ? a : 0.1f * a;
          bb = bb > 0.f ? bb : 0.1f * bb;
        }
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(a, bb);
        packed[c] = *reinterpret_cast<const uint32_t*>(&p2);
      }
      uint4* o = reinterpret_cast<uint4*>(out + 32 * vox);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        o[c] = make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;   // block-uniform: every warp saw this tile's commit
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (tid == 0) atomicOr(err, 1);
      mbar_wait(smem_u32(bar), (uint32_t)(it & 1));   // one more bounded wait for the MMAs in flight
      break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

}  // namespace

bool conv32_tc_fits(const int dims[3]) { return dims[0] % CX == 0 && dims[1] % CY == 0; }

void conv32_tc_pack(const float* W, void* Wp, cudaStream_t st) {
  k_pack_w32<<<(27 * 32 * 32 + 255) / 256, 256, 0, st>>>(W, (__nv_bfloat16*)Wp);
}

void conv32_tc(const void* in, const void* Wp, const float* bias, void* out, const int dims[3], const bool per[3],
               bool act, int* err, cudaStream_t st) {
  set_smem(k_conv32_tc<PMFEM_TC_NBUF>, SMEM_TOTAL);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nt = (int64_t)(dims[0] / CX) * (dims[1] / CY) * dims[2];
  const int64_t per_sm = 3 - PMFEM_TC_NBUF;   // resident blocks per SM
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt, per_sm * (sms > 0 ? sms : 1)));
  k_conv32_tc<PMFEM_TC_NBUF><<<grid, 128, SMEM_TOTAL, st>>>((const __nv_bfloat16*)in, (const __nv_bfloat16*)Wp, bias,
                                           (__nv_bfloat16*)out, dims[0], dims[1], dims[2], per[0], per[1], per[2],
                                           act ? 1 : 0, err);
}

}  // namespace pmfem
