// Device-side data of one handle and the kernel launchers (internal to libpmfem).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

namespace pmfem {

// Opt a kernel into more than 48 KB of dynamic shared memory, once per (kernel, device):
// the call is not a stream operation, so it is made before any graph capture replays it.
template <typename K>
inline void set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::pair<const void*, int> key{(const void*)kernel, dev};
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(key)) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    done.insert(key);
}

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// bfloat16 storage of an operator value: the upper 16 bits of the FP32 number
// (BF16-split precision stores the large operators this way and computes in FP32)
struct bf16_t {
  uint16_t bits;
};

// Vector width of the precorrection's and the projection's SELL layout (values per lane and
// step); the layout builder and the kernels read the same setting.
#ifndef PMFEM_COR_VW
#define PMFEM_COR_VW 8
#endif

// internal magnetisation / state vectors: (x, y, z, pad), one aligned load per gather
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

// Programmatic dependent launch on the evaluation's main stream (PMFEM_PDL 1): each kernel of
// the chain is launched with programmatic stream serialisation, so that it is launched while the
// previous kernel's last blocks run; it waits (griddepcontrol.wait: the previous grid complete,
// its writes visible) before it reads or writes anything, and lets its own successor launch as
// soon as each of its blocks has started.  Without the attribute both instructions do nothing.
// Measured on the 1M-node wire (replayed RK4 graphs): FP32 2.456 -> 2.451 ms per step,
// BF16-split 1.89e9 -> 1.93e9 node-field-evals/s, FP64 2.32e8 -> 2.30e8.
#ifndef PMFEM_PDL
#define PMFEM_PDL 1
#endif
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  if (PMFEM_PDL) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
  } else {
#ifdef __CUDACC__
    kernel<<<grid, block, smem, st>>>(((KArgs)args)...);
#endif
  }
}

// Optional per-launch timing: the handle records a CUDA event pair around each kernel.
enum KernelId : int { KID_CHARGES = 0, KID_ANTERP, KID_FFT_X_FWD, KID_FFT_Y_FWD, KID_FFT_Z_CONV, KID_FFT_Y_INV,
                      KID_FFT_X_INV, KID_INTERP, KID_FIELD, KID_MEMSET, KID_PERM, KID_STENCIL,
                      // surrogate network: the 1 -> 32 layer, the two 32 -> 32 layers, the 32 -> 1 layer
                      KID_SUR_IN, KID_SUR_HIDDEN, KID_SUR_OUT, KID_COUNT };
struct ProfHook {
  void (*fn)(void* ctx, int id, int phase, cudaStream_t st) = nullptr;
  void* ctx = nullptr;
  void begin(int id, cudaStream_t st) const {
    if (fn) fn(ctx, id, 0, st);
  }
  void end(int id, cudaStream_t st) const {
    if (fn) fn(ctx, id, 1, st);
  }
};

// A sparse operator in SELL-32: thread t handles row map[t] (t itself when map is null);
// its element j sits at off[t / 32] + 32 j + t % 32 with column base[t] + delta modulo the
// column count (delta 16-bit when col16) and values val[c][...] (or bval[c][...], stored as
// bfloat16, when that pointer is set); rows of a chunk are padded to its longest.
template <typename T>
struct DevSell {
  int64_t rows = 0;
  const int32_t* map = nullptr;
  const int32_t* len = nullptr;
  const int32_t* base = nullptr;
  const int64_t* off = nullptr;
  const void* delta = nullptr;
  bool col16 = true;
  const T* val[10] = {};
  const bf16_t* bval[10] = {};
};

// Local anisotropy terms (internal order): unknown i has grains grain[ptr[i] .. ptr[i+1]) with
// volume shares w; grain g's row of tab holds its axes a1, a2, a3 (9), c1 = -2 K1 / (mu0 Ms),
// the uniaxial axis u (3), cu = 2 Ku / (mu0 Ms) and two pads.  ptr null: no anisotropy.
constexpr int kGrainTab = 16;
template <typename T>
struct LocalTerms {
  const int32_t* ptr = nullptr;
  const int32_t* grain = nullptr;
  const T* w = nullptr;
  const T* tab = nullptr;
};

// Operator values, grid set-up and work buffers of one precision, all device memory,
// in the internal (box-sorted) order of the unknowns.
template <typename T>
struct DevOps {
  using C2 = typename Vec2<T>::type;
  int64_t Np = 0, nnz = 0, nnzC = 0, nnzX = 0;
  int p = 3, nb = 3;
  int dims[3] = {0, 0, 0}, fft[3] = {0, 0, 0};
  bool periodic[3] = {false, false, false};
  int TY = 1, TZ = 1, pl = 1, pr = 2;
  const int32_t* perm = nullptr;                  // internal -> user unknown
  // sparse operators in SELL-32 (see DevSell)
  DevSell<T> adj;   // components: W^q x,y,z (Ms), E x,y,z (Ms), gradient x,y,z, exchange
  DevSell<T> cor;   // point precorrection
  DevSell<T> pro;   // projection P^T (rows = grid points)
  int64_t nx_exc = 0;                             // projection exceptions
  const int32_t* xnode = nullptr;
  const int64_t* xgrid = nullptr;
  const T* xw = nullptr;
  // near-element entries beyond the pattern
  const int32_t* rowptrX = nullptr;
  const int32_t* colX = nullptr;
  const T* valX = nullptr;                        // nnzX x 3
  // stencils and spectrum
  const int32_t* base = nullptr;                  // Np x 3
  const T* frac = nullptr;                        // Np x 3
  const T* ghat = nullptr;                        // (F0/2+1)(F1/2+1)(F2/2+1), scaled by 1/(F0 F1 F2)
  const C2* tw[3] = {nullptr, nullptr, nullptr};  // exp(-2 pi i j / F_a), j < F_a
  // work buffers
  T* q = nullptr;
  T* e = nullptr;
  T* grid = nullptr;                              // N0 N1 N2 real (Q, then U)
  C2* cbuf = nullptr;                             // F2 x F1 x (F0/2+1) complex
  int* flag = nullptr;                            // device error word
  LocalTerms<T> loc;                              // anisotropy (PMFEM_AN), when set
  ProfHook prof;
};

// error word bits
enum : int { FLAG_NONFINITE_IN = 1, FLAG_NONFINITE_OUT = 2, FLAG_LAYOUT = 4 };

// RK4 epilogue of the field kernel (mode 0: plain field output)
struct RkArgs {
  int mode = 0;            // 0 none, 1 intermediate stage, 2 final combination + renormalise
  const void* m0 = nullptr;   // state at the start of the step
  void* mnext = nullptr;      // stage input for the next evaluation (mode 1)
  void* acc = nullptr;        // running sum of b_i k_i
  double cdt = 0;          // m_next = m0 + cdt * k
  double bw = 0;           // acc (+)= bw * k
  int acc_init = 0;        // 1: acc = bw k, 0: acc += bw k
  double dt6 = 0;          // final: m0 + dt6 (acc + k)
  double gam = 0;          // gamma0 / (1 + alpha^2)
  double alpha = 0;
};

// m_user: N' x 3 in the C-ABI unknown order; m: internal 4-vectors
template <typename T> void launch_perm_in(const DevOps<T>& d, const T* m_user, V4<T>* m, cudaStream_t st);
template <typename T> void launch_perm_out(const DevOps<T>& d, const V4<T>* m, T* m_user, cudaStream_t st);
template <typename T> void launch_charges(const DevOps<T>& d, const V4<T>* m, cudaStream_t st);
template <typename T> void launch_anterp(const DevOps<T>& d, cudaStream_t st);
template <typename T> void launch_fft_conv(const DevOps<T>& d, cudaStream_t st);

// The FFT convolution of one grid, or of count grids of one shape (batched: block row y
// works on grid y, whose grid, spectrum-buffer and PGF-spectrum offsets are
// boff[3y], boff[3y + 1], boff[3y + 2]; boff is null for a single grid).
template <typename T>
struct FftArgs {
  using C2 = typename Vec2<T>::type;
  T* grid = nullptr;
  C2* cbuf = nullptr;
  const T* ghat = nullptr;
  const C2* tw[3] = {nullptr, nullptr, nullptr};
  int dims[3] = {0, 0, 0}, fft[3] = {0, 0, 0};
  const int64_t* boff = nullptr;
  unsigned count = 1;
};
template <typename T> void launch_fft(const FftArgs<T>& a, const ProfHook& prof, cudaStream_t st);
// PMFEM_CHECKS builds: every stored row base, column delta, row map, stencil base and projection
// exception
// checked against its bounds on the device (FLAG_LAYOUT in the error word on a failure)
template <typename T> void launch_layout_checks(const DevOps<T>& d, cudaStream_t st);
template <typename T> void launch_interp(const DevOps<T>& d, const V4<T>* m, cudaStream_t st);
// the two halves of launch_interp: precorrection (+ near and touching elements) from q, m, e;
// then the stencil of the grid potential added on top
template <typename T> void launch_precorr(const DevOps<T>& d, const V4<T>* m, cudaStream_t st);
template <typename T> void launch_stencil(const DevOps<T>& d, const V4<T>* m, cudaStream_t st);
// mode 0 writes H in the C-ABI order (N' x 3); RK modes update internal 4-vector buffers
template <typename T>
void launch_field(const DevOps<T>& d, const V4<T>* m, T* H_user, int comps, double hx, double hy, double hz,
                  const RkArgs& rk, cudaStream_t st);


}  // namespace pmfem
