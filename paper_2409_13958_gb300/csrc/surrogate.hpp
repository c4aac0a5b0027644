// Learned surrogate of the FFT convolution (device network; kernels in surrogate.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "device.hpp"

namespace pmfem {

constexpr int kNetC = 32;   // hidden channels
// parameters of the four layers: W[co][ci][3][3][3] then b[co], 1 -> 32 -> 32 -> 32 -> 1
constexpr int64_t kNetParams = (27 * 1 * kNetC + kNetC) + 2 * (27 * kNetC * kNetC + kNetC) + (27 * kNetC + 1);

struct SurrogateNet {
  int dims[3] = {0, 0, 0};
  bool periodic[3] = {false, false, false};
  bool bf16 = false;          // hidden activations stored as bfloat16
  float sq = 1.f, su = 1.f;   // input and output scales
  int64_t V = 0;              // grid points
  std::vector<void*> allocs;
  float* W[4] = {};           // [tap][ci][co]
  float* b[4] = {};
  float* P = nullptr;         // all parameters, device, in the W[tap][ci][co] / b layout (contiguous)
  float* G = nullptr;         // gradients, same layout
  float* M = nullptr;         // Adam moments
  float* S2 = nullptr;
  float* Wt = nullptr;        // flipped weights of one layer (input-gradient convolution)
  void* h[3] = {};            // hidden activations (float or bfloat16), kNetC x V each
  float* gA = nullptr;        // gradient buffers, kNetC x V floats
  float* gB = nullptr;
  float* pred = nullptr;      // V floats
  double* loss = nullptr;     // device accumulator
  int64_t adam_t = 0;
  // RK use (increment form): charges and potential of the first stage of the current step
  float* Q1 = nullptr;
  float* U1 = nullptr;
  float* Ubuf = nullptr;      // network output
  double* err = nullptr;      // device: [sum (U_net - U)^2, sum U^2] of the judged stages
  // tensor-core path (bfloat16 activations on a grid whose x and y are multiples of 8 and 16):
  // hidden activations channels-last [V][32], the two 32 -> 32 layers on tcgen05
  bool tc = false;
  void* Wp[2] = {};           // packed bfloat16 weights of layers 1 and 2
  int* tc_err = nullptr;      // device: set when a tensor-core wait gave up
  // inputs of the two tensor-core layers (h0, h1) once more in the padded layout their TMA
  // loads read, and a tensor map of each
  void* hpad[2] = {};
  alignas(64) unsigned char tmap[2][128] = {};
  ProfHook prof;              // per-layer CUDA-event timing of the forward pass (when enabled)
};

bool conv32_tc_fits(const int dims[3]);
void conv32_tc_pack(const float* W, void* Wp, cudaStream_t st);
// tensor map (128 bytes at tmap) of a padded channels-last bfloat16 buffer of the grid dims
bool conv32_tc_tensor_map(const void* padded, const int dims[3], void* tmap);
// out = act(bias + conv(in)) with in read through its tensor map (its padded copy); out
// channels-last [V][32], and also written padded to pout when pout is not null
void conv32_tc(const void* tmap, const void* Wp, const float* bias, void* out, void* pout, const int dims[3],
               const bool per[3], bool act, int* err, cudaStream_t st);

#ifdef __CUDACC__
// Padded layout of a tensor-core layer's input: four planes of 8 bfloat16 channels, each of
// (X + 2)(Y + 2)(Z + 2) voxels, [group][z][y][x][8], the outer layer holding periodic copies
// along periodic axes and zeros along open ones.  pad_slots lists the padded voxels that hold
// voxel (x, y, z): itself and, on a periodic border, its copies (up to 8 at a corner).
__device__ __forceinline__ int pad_slots(int x, int y, int z, int X, int Y, int Z, bool px, bool py, bool pz,
                                         int64_t slot[8]) {
  int xs[2] = {x + 1, 0}, ys[2] = {y + 1, 0}, zs[2] = {z + 1, 0};
  int nx = 1, ny = 1, nz = 1;
  if (px && x == 0) xs[nx++] = X + 1;
  else if (px && x == X - 1) xs[nx++] = 0;
  if (py && y == 0) ys[ny++] = Y + 1;
  else if (py && y == Y - 1) ys[ny++] = 0;
  if (pz && z == 0) zs[nz++] = Z + 1;
  else if (pz && z == Z - 1) zs[nz++] = 0;
  int n = 0;
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) slot[n++] = xs[a] + (int64_t)(X + 2) * (ys[b] + (int64_t)(Y + 2) * zs[c]);
  return n;
}
#endif

int64_t net_layer_offset(int layer, bool bias);                 // offset in the device layout
int net_create(SurrogateNet& n, const int dims[3], const bool periodic[3], bool bf16, std::string& msg);
void net_destroy(SurrogateNet& n);
// caller order (W[co][ci][dz][dy][dx], b per layer) <-> device layout (host copies)
void net_params_to_device_layout(const float* in, std::vector<float>& out);
void net_params_from_device_layout(const float* in, std::vector<float>& out);
void net_forward(SurrogateNet& n, const float* Q, float* U, cudaStream_t st);
// gradient of the mean squared error of one pair, added into n.G; loss added into *n.loss
void net_backward(SurrogateNet& n, const float* Q, const float* U, cudaStream_t st);
void net_adam(SurrogateNet& n, float lr, int64_t t, cudaStream_t st);
// U = U1 + net(Q - Q1), Q and U on the same grid buffer (Q in, U out); tmp holds V floats
void net_increment(SurrogateNet& n, float* grid, cudaStream_t st);
// accumulate |net(Q - Q1) + U1 - U|^2 and |U|^2 for a judged stage (grid holds U, Qs the stage's Q)
void net_judge(SurrogateNet& n, const float* Qs, const float* U, cudaStream_t st);

}  // namespace pmfem
