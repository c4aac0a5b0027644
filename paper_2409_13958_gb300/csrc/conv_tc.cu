// 32 -> 32 channel 3x3x3 convolution of the surrogate network on the 5th-generation tensor
// cores (tcgen05): an implicit GEMM D[128 voxels][32 out] = sum over 27 taps of
// A_tap[128 voxels][32 in] * W_tap[32 out][32 in]^T, BF16 operands in shared memory, FP32
// accumulator in tensor memory.
//
// A tile is 8 (x) x 16 (y) x 2 (z) output voxels: 128 MMA rows (x, y) and two z planes, whose
// accumulators sit side by side in 64 TMEM columns (plane 0 in 0-31, plane 1 in 32-63).  Its
// input halo (10 x 18 x 4 voxels) sits in shared memory as [channel group][z][y][x][8
// channels], so that the 8 channels of one voxel are one 16-byte row: for taps (dx, dy) and
// halo plane w the A operand of an MMA is the halo seen from offset (dx, dy, w) -- 8
// consecutive x voxels form one 8 x 16-byte core matrix, the 16 y rows of the tile sit 10
// voxels apart (stride-dimension offset 160 B), and the next 8 channels sit one channel-group
// block further (leading-dimension offset).  No im2col copy is made.
//
// Halo plane w feeds output plane 0 through tap dz = w and output plane 1 through tap dz = w - 1.
// The weights are packed per (dy, dx, channel group) as three 32-row blocks in the order dz = 2,
// 1, 0, so that for w = 1 and w = 2 the blocks of (dz = w, dz = w - 1) are adjacent: one MMA of
// N = 64 computes both planes' contributions of that halo plane.  w = 0 and w = 3 feed one plane
// each (N = 32).  Per (dy, dx) and 16-channel half: two MMAs of N = 64 and two of N = 32, which
// measured 48 and 46 cycles each on GB300 (N = 32 runs at a third of the tensor peak, N = 64 at
// two thirds), against six of N = 32 for the two planes apart.
//
// One persistent block per SM, warp-specialised: a producer warp loads the halos of the block's
// tiles with TMA (4 tensor copies, one per 8-channel group) into a ring of three
// shared-memory stages; one thread of the MMA warp issues a tile's 72 MMAs into one of two TMEM
// accumulator pairs and commits them to the stage's "empty" and the pair's "full" barrier; four
// epilogue warps drain a finished pair (tcgen05.ld), release it, add the bias, apply the
// activation and store.  TMA loads, MMAs and the epilogue of different tiles overlap.
//
// The input is read through a tensor map over its padded, group-planar copy ([4 groups][Z + 2]
// [Y + 2][X + 2][8 channels], periodic copies in the outer layer: TMA does not wrap), so every
// halo is one in-range box per group whose rows are 160 contiguous bytes.  The output is
// channels-last BF16, [voxel][32], and optionally also written in the padded layout.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <utility>

#include "device.hpp"
#include "surrogate.hpp"

namespace pmfem {
namespace {

constexpr int CX = 8, CY = 16, CZ = 2;               // output tile (x, y, z)
constexpr int HX = CX + 2, HY = CY + 2, HZ = CZ + 2; // halo
constexpr int PLANE_S = HY * HX * 16;                // 2880 B: one z plane of one channel group
constexpr int CG_S = HZ * PLANE_S;                   // 11520 B: one channel group (LBO of A)
constexpr int SMEM_X = 4 * CG_S;                     // 46080 B per halo stage
constexpr int TMA_BYTES = SMEM_X;                    // loaded per stage
constexpr int WBLK = 32 * 16;                        // one 32-row weight block of 8 inputs: 512 B
constexpr int WCG_S = 3 * WBLK;                      // the three dz blocks of one (dy, dx, group)
constexpr int SMEM_W = 9 * 4 * WCG_S;                // 55296 B
constexpr int NSTAGE = 3;                            // halo stages
constexpr int NACC = 2;                              // TMEM accumulator pairs (2 x 64 columns)
constexpr int TMEM_COLS = 128;
constexpr int PROD_WARP = 0;                         // TMA issue (one lane)
constexpr int MMA_WARP = 1;                          // allocates TMEM; one lane issues
constexpr int EPI0 = 2;                              // epilogue warps 2-5 (TMEM lane quarters 2, 3, 0, 1)
constexpr int NTHREADS = (EPI0 + 4) * 32;            // 192
// barriers: full[NSTAGE], empty[NSTAGE], afull[NACC], aempty[NACC], done; then the TMEM address
// and the abort word; 128 more bytes to align the stages to 128 B
constexpr int NBAR = 2 * NSTAGE + 2 * NACC + 1;
constexpr int SMEM_TOTAL = 128 + SMEM_W + NSTAGE * SMEM_X + NBAR * 8 + 16;
// Every descriptor this kernel forms stays inside s_w and its halo stage.  A: the largest start
// is halo plane 3 with dy = dx = 2 in the second 16-channel half, 3 PLANE_S + 22 x 16 + 2 CG_S,
// plus one more K core matrix (CG_S), 15 row groups of 160 B and one core matrix of 128 B; the
// rows of one plane stay inside it ((2 + 15) x 160 + (2 + 7) x 16 + 16 = PLANE_S).
// B: the largest start is (dy, dx) = (2, 2), group 2, block dz = 0, plus one more K core matrix
// (WCG_S) and 32 rows (512 B), which ends exactly at SMEM_W.
static_assert(3 * PLANE_S + (2 * HX + 2) * 16 + 2 * CG_S + CG_S + 15 * HX * 16 + 128 == SMEM_X, "A extent");
static_assert((2 + 15) * HX * 16 + (2 + 7) * 16 + 16 == PLANE_S && CG_S % 128 == 0, "plane");
static_assert((8 * 4 + 2) * WCG_S + 2 * WBLK + WCG_S + WBLK == SMEM_W, "B extent");
static_assert(SMEM_X % 128 == 0 && SMEM_W % 128 == 0, "stage alignment");
static_assert(SMEM_TOTAL <= 227 * 1024, "shared memory");
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
__host__ __device__ constexpr uint32_t idesc_n(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// MMA number I of a tile: group g = I / 4 is (dy, dx, 16-channel half) = (g / 6, g / 2 % 3, g % 2);
// k = I % 4 takes halo plane w = 0 (N = 32 into plane 0), w = 3 (N = 32 into plane 1), w = 1 and
// w = 2 (N = 64 into both).  The first group's two N = 32 MMAs start the accumulators; every
// later MMA accumulates.  Offsets are immediates added inside the asm (the descriptors' address
// fields are byte addresses >> 4); one elected lane of the converged warp issues.
template <int I>
__device__ __forceinline__ void mma_one(uint32_t acc, uint64_t adesc0, uint64_t bdesc0) {
  constexpr int g = I / 4, k = I % 4;
  constexpr int dy = g / 6, dx = (g / 2) % 3, half = g % 2;
  constexpr int w = k == 0 ? 0 : k == 1 ? 3 : k - 1;
  constexpr int blk = w == 0 ? 2 : w == 3 ? 0 : 2 - w;   // block order dz = 2, 1, 0
  constexpr int aoff = (w * PLANE_S + (dy * HX + dx) * 16 + half * 2 * CG_S) >> 4;
  constexpr int boff = (((dy * 3 + dx) * 4 + half * 2) * WCG_S + blk * WBLK) >> 4;
  constexpr int col = w == 3 ? 32 : 0;
  constexpr uint32_t idesc = idesc_n(k < 2 ? 32u : 64u);
  constexpr int accum = I < 2 ? 0 : 1;
  asm volatile(
      "{\n .reg .pred p, e;\n .reg .b32 rx, ta, id, ac;\n .reg .b64 ad, bd;\n"
      " add.s64 ad, %1, %3;\n add.s64 bd, %2, %4;\n add.u32 ta, %0, %5;\n"
      " mov.u32 id, %6;\n mov.u32 ac, %7;\n setp.ne.u32 p, ac, 0;\n"
      " elect.sync rx|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [ta], ad, bd, id, p;\n}\n" ::"r"(acc),
      "l"(adesc0), "l"(bdesc0), "n"(aoff), "n"(boff), "n"(col), "n"(idesc), "n"(accum));
}
template <int... I>
__device__ __forceinline__ void mma_tile(uint32_t acc, uint64_t adesc0, uint64_t bdesc0,
                                         std::integer_sequence<int, I...>) {
  (mma_one<I>(acc, adesc0, bdesc0), ...);
}

__device__ __forceinline__ void commit_elect(uint32_t bar) {
  asm volatile(
      "{\n .reg .pred e;\n .reg .b32 rx;\n elect.sync rx|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
      : "memory");
}

// W[tap][ci][co] (FP32) -> Wp[dy][dx][ci / 8][block of dz: 2, 1, 0][co][ci % 8] (BF16)
__global__ void k_pack_w32(const float* __restrict__ W, __nv_bfloat16* __restrict__ Wp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 27 * 32 * 32) return;
  const int tap = k >> 10, r = k & 1023, ci = r >> 5, co = r & 31;
  const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
  Wp[((((dy * 3 + dx) * 4 + (ci >> 3)) * 3 + (2 - dz)) * 32 + co) * 8 + (ci & 7)] = __float2bfloat16_rn(W[k]);
}

struct TileXYZ {
  int x0, y0, z0;
};
__device__ __forceinline__ TileXYZ tile_origin(int tile, int X, int Y) {
  const int ntx = X / CX, nty = Y / CY;
  return {(tile % ntx) * CX, ((tile / ntx) % nty) * CY, (tile / (ntx * nty)) * CZ};
}

// The halo of a tile: 4 TMA loads, one per channel group, of box (10 x 8 channels, 18 y, 4 z)
// from the group-planar padded input (rows of 160 contiguous bytes), whose padded coordinates
// (x0, y0, z0) are the halo's origin (all in range; x in elements, 8 x0, so 16-byte aligned);
// each lands dense as [hz][hy][hx][8] in its group's block and completes on the stage's barrier.
__device__ __forceinline__ void tma_halo(uint32_t stage, const CUtensorMap* tmap, int tile, int X, int Y,
                                         uint32_t bar) {
  const TileXYZ o = tile_origin(tile, X, Y);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "n"(TMA_BYTES) : "memory");
#pragma unroll
  for (int cg = 0; cg < 4; ++cg)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(stage + (uint32_t)(cg * CG_S)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(8 * o.x0), "r"(o.y0), "r"(o.z0), "r"(cg), "r"(bar)
        : "memory");
}

// Every wait is bounded: a wait that gives up sets the block's abort word and the error word,
// and every role leaves its loop at the next tile; before TMEM is freed the MMA warp waits
// (bounded) for its last MMAs and the producer for its last loads.
__global__ void __launch_bounds__(NTHREADS, 1) k_conv32_tc(const __grid_constant__ CUtensorMap tmap,
                                                           const __nv_bfloat16* __restrict__ Wp,
                                                           const float* __restrict__ bias,
                                                           __nv_bfloat16* __restrict__ out,
                                                           __nv_bfloat16* __restrict__ pout, int X, int Y, int Z,
                                                           bool px, bool py, bool pz, int act,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);   // 128-B aligned
  uint4* s_w = reinterpret_cast<uint4*>(smem);
  const uint32_t xs0 = smem_u32(smem + SMEM_W);            // stage s at xs0 + s * SMEM_X
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SMEM_W + NSTAGE * SMEM_X);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_w = reinterpret_cast<volatile int*>(tslot + 1);
  const uint32_t b0 = smem_u32(bars);
  auto full = [&](int s) { return b0 + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return b0 + 8u * (uint32_t)(NSTAGE + s); };
  auto afull = [&](int a) { return b0 + 8u * (uint32_t)(2 * NSTAGE + a); };
  auto aempty = [&](int a) { return b0 + 8u * (uint32_t)(2 * NSTAGE + NACC + a); };
  const uint32_t done = b0 + 8u * (uint32_t)(2 * NSTAGE + 2 * NACC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (X / CX) * (Y / CY) * (Z / CZ);
  const unsigned FULLMASK = 0xffffffffu;

  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full(s)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty(s)));
    }
    for (int a = 0; a < NACC; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(afull(a)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(aempty(a)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done));
    *abort_w = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
  }
  // the weights, once per block (16-byte loads and stores), visible to the tensor cores
  const uint4* wg = reinterpret_cast<const uint4*>(Wp);
  for (int k = tid; k < SMEM_W / 16; k += NTHREADS) s_w[k] = wg[k];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  auto give_up = [&]() {
    *abort_w = 1;
    atomicOr(err, 1);
  };

  if (warp == PROD_WARP) {
    // producer: the whole warp walks the tiles and waits, lane 0 issues the loads
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !__any_sync(FULLMASK, *abort_w); tile += gridDim.x, ++it) {
      const int s = it % NSTAGE, u = it / NSTAGE;
      if (!__all_sync(FULLMASK, u == 0 || mbar_wait(empty(s), (uint32_t)((u - 1) & 1)))) {
        if (lane == 0) give_up();
        break;
      }
      if (lane == 0) tma_halo(xs0 + (uint32_t)(s * SMEM_X), &tmap, tile, X, Y, full(s));
      __syncwarp();
    }
    // the loads of the last stages have landed before the block can exit (each of those
    // phases is the barrier's latest, so the wait also succeeds once the MMA warp consumed it)
    for (int j = it - 1; j >= 0 && j >= it - NSTAGE; --j)
      if (!__all_sync(FULLMASK, mbar_wait(full(j % NSTAGE), (uint32_t)((j / NSTAGE) & 1))) && lane == 0) give_up();
  } else if (warp == MMA_WARP) {
    // the whole warp walks the tiles and waits; one elected lane issues the MMAs and commits
    const uint64_t bdesc0 = smem_desc(smem_u32(s_w), WCG_S, 8 * 16);
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !__any_sync(FULLMASK, *abort_w); tile += gridDim.x, ++it) {
      const int s = it % NSTAGE, a = it % NACC;
      const bool ok = __all_sync(FULLMASK, mbar_wait(full(s), (uint32_t)((it / NSTAGE) & 1)) &&
                                               (it < NACC || mbar_wait(aempty(a), (uint32_t)((it / NACC - 1) & 1))));
      if (!ok) {
        if (lane == 0) give_up();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t adesc0 = smem_desc(xs0 + (uint32_t)(s * SMEM_X), CG_S, HX * 16);
      mma_tile(tmem + (uint32_t)(a * 64), adesc0, bdesc0, std::make_integer_sequence<int, 72>{});
      // the halo stage is free, and the accumulator pair full, once these MMAs complete
      commit_elect(empty(s));
      commit_elect(afull(a));
    }
    // every MMA this warp issued has completed before TMEM is freed
    commit_elect(done);
    if (!__all_sync(FULLMASK, mbar_wait(done, 0u)) && lane == 0) give_up();
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ... + 31, i.e. rows m of both planes
    const int q = warp & 3, m = 32 * q + lane;
    const uint32_t lanebase = (uint32_t)(32 * q) << 16;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles && !__any_sync(FULLMASK, *abort_w); tile += gridDim.x, ++it) {
      const int a = it % NACC;
      if (!__all_sync(FULLMASK, mbar_wait(afull(a), (uint32_t)((it / NACC) & 1)))) {
        if (lane == 0) give_up();   // warp-uniform: tcgen05.ld below needs the whole warp
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r[CZ][32];
#pragma unroll
      for (int t = 0; t < CZ; ++t) {
        const uint32_t taddr = tmem + lanebase + (uint32_t)(a * 64 + t * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[t][0]), "=r"(r[t][1]), "=r"(r[t][2]), "=r"(r[t][3]), "=r"(r[t][4]), "=r"(r[t][5]),
              "=r"(r[t][6]), "=r"(r[t][7]), "=r"(r[t][8]), "=r"(r[t][9]), "=r"(r[t][10]), "=r"(r[t][11]),
              "=r"(r[t][12]), "=r"(r[t][13]), "=r"(r[t][14]), "=r"(r[t][15]), "=r"(r[t][16]), "=r"(r[t][17]),
              "=r"(r[t][18]), "=r"(r[t][19]), "=r"(r[t][20]), "=r"(r[t][21]), "=r"(r[t][22]), "=r"(r[t][23]),
              "=r"(r[t][24]), "=r"(r[t][25]), "=r"(r[t][26]), "=r"(r[t][27]), "=r"(r[t][28]), "=r"(r[t][29]),
              "=r"(r[t][30]), "=r"(r[t][31])
            : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // the pair is drained: the MMA warp may fill it with a later tile
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(aempty(a));
      const TileXYZ o = tile_origin(tile, X, Y);
#pragma unroll
      for (int t = 0; t < CZ; ++t) {
        const int x = o.x0 + (m & 7), y = o.y0 + (m >> 3), z = o.z0 + t;
        uint4 v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t pk[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int ch = 8 * c + 2 * j;
            float v0 = __uint_as_float(r[t][ch]) + bias[ch];
            float v1 = __uint_as_float(r[t][ch + 1]) + bias[ch + 1];
            if (act) {
              v0 = v0 > 0.f ? v0 : 0.1f * v0;
              v1 = v1 > 0.f ? v1 : 0.1f * v1;
            }
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(v0, v1);
            pk[j] = *reinterpret_cast<const uint32_t*>(&p2);
          }
          v[c] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + 32 * (x + (int64_t)X * (y + (int64_t)Y * z)));
#pragma unroll
        for (int c = 0; c < 4; ++c) dst[c] = v[c];
        if (pout) {
          int64_t slot[8];
          const int ns = pad_slots(x, y, z, X, Y, Z, px, py, pz, slot);
          const int64_t vp = (int64_t)(X + 2) * (Y + 2) * (Z + 2);
          for (int k = 0; k < ns; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) reinterpret_cast<uint4*>(pout)[c * vp + slot[k]] = v[c];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
}

}  // namespace

bool conv32_tc_fits(const int dims[3]) { return dims[0] % CX == 0 && dims[1] % CY == 0 && dims[2] % CZ == 0; }

void conv32_tc_pack(const float* W, void* Wp, cudaStream_t st) {
  k_pack_w32<<<(27 * 32 * 32 + 255) / 256, 256, 0, st>>>(W, (__nv_bfloat16*)Wp);
}

bool conv32_tc_tensor_map(const void* padded, const int dims[3], void* tmap) {
  // cuTensorMapEncodeTiled, reached through the runtime (no link against the driver library)
  using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<EncodeTiled>(fn);
  }
  // group-planar padded layout [4][Z + 2][Y + 2][X + 2][8]: dims (8 (X + 2) elements, Y + 2, Z + 2, 4
  // groups), strides of dims 1-3 in bytes
  const cuuint64_t X2 = (cuuint64_t)dims[0] + 2, Y2 = (cuuint64_t)dims[1] + 2, Z2 = (cuuint64_t)dims[2] + 2;
  const cuuint64_t gdim[4] = {8 * X2, Y2, Z2, 4};
  const cuuint64_t gstride[3] = {16 * X2, 16 * X2 * Y2, 16 * X2 * Y2 * Z2};
  const cuuint32_t box[4] = {8 * HX, HY, HZ, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return encode(reinterpret_cast<CUtensorMap*>(tmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(padded),
                gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void conv32_tc(const void* tmap, const void* Wp, const float* bias, void* out, void* pout, const int dims[3],
               const bool per[3], bool act, int* err, cudaStream_t st) {
  set_smem(k_conv32_tc, SMEM_TOTAL);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nt = (int64_t)(dims[0] / CX) * (dims[1] / CY) * (dims[2] / CZ);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt, sms > 0 ? sms : 1));
  k_conv32_tc<<<grid, NTHREADS, SMEM_TOTAL, st>>>(*reinterpret_cast<const CUtensorMap*>(tmap),
                                                 (const __nv_bfloat16*)Wp, bias, (__nv_bfloat16*)out,
                                                 (__nv_bfloat16*)pout, dims[0], dims[1], dims[2], per[0], per[1],
                                                 per[2], act ? 1 : 0, err);
}

}  // namespace pmfem
