// Launchers of the implicit midpoint step's node-local kernels and reductions (implicit.cu);
// the Newton and Krylov loops that call them are in api.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pmfem {

constexpr int kMaxKrylov = 64;   // longest GMRES cycle (restart length) the kernels take
constexpr int kImpBlocks = 1024; // blocks of a reduction (fixed, so its sums run in a fixed order)

// up to kMaxKrylov + 1 device vectors passed by value to one launch
template <typename T>
struct VecList {
  const T* p[kMaxKrylov + 1] = {};
};

template <typename T> void imp_mid(int64_t n, const T* m0, const T* y, T* mb, cudaStream_t st);
template <typename T>
void imp_residual(int64_t n, const T* m0, const T* y, const T* mb, const T* H, double dt, double g, double alpha,
                  T* R, cudaStream_t st);
template <typename T>
void imp_jvp(int64_t n, const T* mb, const T* H, const T* Av, const T* v, double dt, double g, double alpha, T* out,
             cudaStream_t st);
template <typename T>
void imp_blocks(int64_t n, const T* mb, const T* H, const T* c, double dt, double g, double alpha, T* Pinv,
                cudaStream_t st);
template <typename T> void imp_apply_blocks(int64_t n, const T* Pinv, const T* x, T* out, cudaStream_t st);
// out[j] = V_j . w for j < cnt (FP64; partial holds nblocks * cnt doubles)
template <typename T>
void imp_multidot(int64_t len, const VecList<T>& V, int cnt, const T* w, double* partial, int nblocks, double* out,
                  cudaStream_t st);
// w = a w + csign sum_j coef[j] V_j  (coef: cnt device doubles, e.g. the output of imp_multidot)
template <typename T>
void imp_combine(int64_t len, const VecList<T>& V, int cnt, const double* coef, double csign, double a, T* w,
                 cudaStream_t st);
// out = w / sqrt(*n2), n2 a device scalar (zero when it is not positive)
template <typename T>
void imp_scale_invnorm(int64_t len, const T* w, const double* n2, T* out, cudaStream_t st);

}  // namespace pmfem
