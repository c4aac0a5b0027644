// Handle of one mesh (pmfem_t): the host set-up, the device data of the current precision
// and the per-launch timing records.  Shared by the C-ABI (api.cu) and the batch (batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pmfem.h"
#include "device.hpp"
#include "internal.hpp"
#include "surrogate.hpp"

struct pmfem_state {
  using Setup = pmfem::Setup;
  using Error = pmfem::Error;
  Setup s;
  Error err;
  int prec = PMFEM_FP64;
  int bf16_ops = PMFEM_BF16_PRECORRECTION | PMFEM_BF16_PROJECTION | PMFEM_BF16_GRADIENT;
  double hap[3] = {0, 0, 0};
  // device side
  bool dev_ready = false;
  int dev_prec = -1;
  cudaStream_t stream = nullptr;
  // the precorrection runs on `side` while the projection and FFT run on the caller's stream:
  // ev_fork (after the charges) and ev_join (after the precorrection) order the two
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<void*> allocs;
  pmfem::DevOps<double> d64;
  pmfem::DevOps<float> d32;
  void* m = nullptr;      // internal state, N' 4-vectors in the internal order
  void* mA = nullptr;     // RK stage buffers (4-vectors)
  void* mB = nullptr;
  void* acc = nullptr;
  void* mF = nullptr;     // permuted input of pmfem_field (4-vectors)
  void* hin = nullptr;    // N' x 3 user-order staging for the host-buffer calls
  void* hout = nullptr;
  int* flag = nullptr;
  // device address of the library's fixed scratch array for pmfem_field_noalloc, looked up
  // whenever the device data are (re)built, in the context that holds them
  void* noalloc_base = nullptr;
  std::string noalloc_why;
  // implicit midpoint steps: work vectors (N' x 3), preconditioner blocks, exchange diagonal,
  // reduction scratch; device memory of the handle (freed with the device data)
  std::vector<void*> imp_vec;
  void* imp_pinv = nullptr;
  void* imp_c = nullptr;
  void* imp_red = nullptr;
  int imp_prec = -1;
  // Bloch-phase convolution: the spectrum of the last k0 (device, precision of the handle)
  // and three complex scratch grids
  void* bloch_spec = nullptr;
  void* bloch_buf[3] = {nullptr, nullptr, nullptr};
  double bloch_k0[3] = {0, 0, 0};
  int bloch_prec = -1;
  // per-launch timing (pmfem_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  struct Rec { int id; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  int open_id[pmfem::KID_COUNT] = {};
  cudaEvent_t open_ev[pmfem::KID_COUNT] = {};
  int64_t prof_count[pmfem::KID_COUNT] = {};
  double prof_ms[pmfem::KID_COUNT] = {};
  int64_t dev_info[13] = {};   // layout facts of the current device upload
  // one RK4 step captured as a CUDA graph (pmfem_llg_step without timing or surrogate)
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  // learned surrogate of the FFT convolution (pmfem_surrogate_*)
  pmfem::SurrogateNet* net = nullptr;
  int sur_every = 0;            // 0: off; k: full P-AIM (judged) on every k-th RK step
  int64_t sur_step = 0, sur_evals = 0, sur_judged = 0;
};
