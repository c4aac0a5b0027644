// Set-up on the GPU, in FP64 (pmfem_set_setup_device): the three set-up stages whose
// arithmetic grows with the mesh and the grid run as CUDA kernels on the current device.
//   K10  PGF spectrum (Eq. 15 on the grid of Eq. 16, BAIM step 2): G^p at every distinct grid
//        offset by the Ewald-type sums, then the separable even-cosine transform per axis.
//   K11a near-element correction (Eq. 14c): exact element integrals minus nodal point charges
//        for every near placement, one thread per observer row (placements planned on the host).
//   K11b point precorrection (BAIM step 4): for every box-near source image, G0 minus what the
//        grid carries; one warp per observer row enumerates its sources, sorts them by column
//        and evaluates the entries.
// The formulas are the ones of the host set-up (setup_math.hpp, compiled for both sides) and
// every sum runs in the host's order, so the two set-ups agree to the last bits of the
// device's and the host's libm.  Results are copied back into the host set-up (s.ghat, the
// near-element values, s.C), from which the device layout is built as before.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.hpp"
#include "setup_math.hpp"

namespace pmfem {
namespace {

struct DBuf {
  void* p = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

int cuda_fail(Error& err, const char* what, cudaError_t e) {
  err = {ECUDA_, std::string("GPU set-up: ") + what + ": " + cudaGetErrorString(e)};
  return ECUDA_;
}

#define SG_CK(what, x)                               \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(err, what, e_); \
  } while (0)

int dalloc(DBuf& b, size_t bytes, Error& err) {
  cudaError_t e = cudaMalloc(&b.p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    b.p = nullptr;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      err = {ENOMEM_, "GPU set-up: device allocation of " + std::to_string(bytes) + " bytes failed"};
      return ENOMEM_;
    }
    return cuda_fail(err, "cudaMalloc", e);
  }
  return OK;
}

template <typename T>
int dput(DBuf& b, const T* h, size_t n, Error& err) {
  int rc = dalloc(b, n * sizeof(T), err);
  if (rc) return rc;
  if (n) SG_CK("copy to device", cudaMemcpy(b.p, h, n * sizeof(T), cudaMemcpyHostToDevice));
  return OK;
}

int grid_for(int64_t n, int threads) { return (int)std::min<int64_t>((n + threads - 1) / threads, 1 << 30); }

// ------------------------------------------------------------------ K10
__global__ void k_pgf_offsets(sm::PgfParams P, double d0, double d1, double d2, int U0, int U1, int64_t n,
                              double* __restrict__ Ku) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t dx = i % U0, dy = (i / U0) % U1, dz = i / ((int64_t)U0 * U1);
  Ku[i] = (!dx && !dy && !dz) ? P.reg0 : sm::pgf_eval(P, dx * d0, dy * d1, dz * d2);
}

// out[c with c[axis] = k] = sum_d tab[k][d] in[c with c[axis] = d]  (shape s -> s with K on axis)
__global__ void k_cos_axis(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ tab,
                           int s0, int s1, int s2, int axis, int K, int64_t nout) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nout) return;
  const int ns0 = axis == 0 ? K : s0, ns1 = axis == 1 ? K : s1;
  int64_t c[3] = {i % ns0, (i / ns0) % ns1, i / ((int64_t)ns0 * ns1)};
  const int64_t kk = c[axis];
  c[axis] = 0;
  const int64_t st[3] = {1, s0, (int64_t)s0 * s1};
  const int S = axis == 0 ? s0 : axis == 1 ? s1 : s2;
  const int64_t off = c[0] * st[0] + c[1] * st[1] + c[2] * st[2];
  const double* row = tab + kk * S;
  double acc = 0;
  for (int d = 0; d < S; ++d) acc += row[d] * in[off + d * st[axis]];
  out[i] = acc;
}

// ------------------------------------------------------------------ K11a
__global__ void k_near_rows(sm::NearArgs A, int64_t Np, double* __restrict__ out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= Np) return;
  sm::near_eval_row(A, n, out);
}

// ------------------------------------------------------------------ K11b
struct PrecorrArgs {
  const double* pos_f;    // Np x 3
  const int32_t* base;    // Np x 3
  const double* frac;     // Np x 3
  const int32_t* box;     // Np x 3
  const int64_t* bptr;    // boxes + 1
  const int32_t* bl;      // Np: unknowns box by box
  const double* T0;       // W^3 table of G0' on integer grid offsets
  int R;
  int dimN[3];
  int per[3];
  double L[3];
  int p;
  int nb;
  int64_t Np;
};

// target box of offset (ox, oy, oz) from box b: false outside an open axis; img in periods
__device__ __forceinline__ bool near_box(const PrecorrArgs& A, const int32_t* b, int ox, int oy, int oz, int64_t* bi,
                                         int img[3]) {
  int64_t t[3] = {(int64_t)b[0] + ox, (int64_t)b[1] + oy, (int64_t)b[2] + oz};
  for (int a = 0; a < 3; ++a) {
    img[a] = 0;
    if (A.per[a]) {
      const int64_t q = t[a] >= 0 ? t[a] / A.dimN[a] : -((-t[a] + A.dimN[a] - 1) / A.dimN[a]);
      img[a] = (int)q;
      t[a] -= q * A.dimN[a];
    } else if (t[a] < 0 || t[a] >= A.dimN[a]) {
      return false;
    }
  }
  *bi = t[0] + (int64_t)A.dimN[0] * (t[1] + (int64_t)A.dimN[1] * t[2]);
  return true;
}

__global__ void k_precorr_count(PrecorrArgs A, int32_t* __restrict__ len) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= A.Np) return;
  const int32_t* b = A.box + 3 * n;
  int64_t c = 0;
  for (int oz = -A.nb; oz <= A.nb; ++oz)
    for (int oy = -A.nb; oy <= A.nb; ++oy)
      for (int ox = -A.nb; ox <= A.nb; ++ox) {
        int64_t bi;
        int img[3];
        if (near_box(A, b, ox, oy, oz, &bi, img)) c += A.bptr[bi + 1] - A.bptr[bi];
      }
  len[n] = (int32_t)c;
}

// One warp per row: the row's (source, image) keys go to shared memory, are sorted by source
// (each source appears once per row: the periodic axes have at least 2 near_boxes + 2 boxes),
// and every lane then evaluates entries in sorted order.  S = keys per warp, a power of two.
__global__ void __launch_bounds__(128) k_precorr_fill(PrecorrArgs A, const int64_t* __restrict__ rowptr, int S,
                                                       int32_t* __restrict__ col, double* __restrict__ val) {
  extern __shared__ unsigned long long keys_all[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t n = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (n >= A.Np) return;   // whole warps leave together
  unsigned long long* keys = keys_all + (size_t)wib * S;
  const int64_t r0 = rowptr[n];
  const int len = (int)(rowptr[n + 1] - r0);
  const int32_t* b = A.box + 3 * n;
  // enumerate: box offsets split over the lanes, slots by a warp-wide running count
  const int side = 2 * A.nb + 1, noff = side * side * side;
  int filled = 0;
  for (int o0 = 0; o0 < noff; o0 += 32) {
    const int o = o0 + lane;
    int64_t bi = 0, cnt = 0;
    int img[3] = {0, 0, 0};
    if (o < noff) {
      const int ox = o % side - A.nb, oy = (o / side) % side - A.nb, oz = o / (side * side) - A.nb;
      if (near_box(A, b, ox, oy, oz, &bi, img)) cnt = A.bptr[bi + 1] - A.bptr[bi];
    }
    int incl = (int)cnt;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    const int start = filled + incl - (int)cnt;
    const unsigned code = (unsigned)(img[0] + 1) | ((unsigned)(img[1] + 1) << 2) | ((unsigned)(img[2] + 1) << 4);
    for (int64_t q = 0; q < cnt; ++q) {
      const unsigned long long k = (unsigned long long)(unsigned)A.bl[A.bptr[bi] + q];
      keys[start + q] = (k << 8) | code;
    }
    filled += __shfl_sync(0xffffffffu, incl, 31);
  }
  for (int i = filled + lane; i < S; i += 32) keys[i] = ~0ull;
  __syncwarp();
  // bitonic sort of the S keys, ascending
  for (int size = 2; size <= S; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane; t < (S >> 1); t += 32) {
        const int lo = 2 * stride * (t / stride) + (t % stride), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long x = keys[lo], y = keys[hi];
        if ((x > y) == up) {
          keys[lo] = y;
          keys[hi] = x;
        }
      }
      __syncwarp();
    }
  // entries
  double wn[3][6];
  for (int a = 0; a < 3; ++a) sm::lagrange(A.frac[3 * n + a], A.p, wn[a]);
  const double* rn = A.pos_f + 3 * n;
  for (int i = lane; i < len; i += 32) {
    const unsigned long long key = keys[i];
    const int32_t k = (int32_t)(key >> 8);
    const unsigned code = (unsigned)(key & 0xffu);
    const int img[3] = {(int)(code & 3u) - 1, (int)((code >> 2) & 3u) - 1, (int)((code >> 4) & 3u) - 1};
    int Db[3];
    for (int a = 0; a < 3; ++a) Db[a] = A.base[3 * n + a] - A.base[3 * (int64_t)k + a];
    const bool self = k == n && !img[0] && !img[1] && !img[2];
    col[r0 + i] = k;
    val[r0 + i] = sm::precorr_value(rn, A.pos_f + 3 * (int64_t)k, img, A.L, Db, wn, A.frac + 3 * (int64_t)k, A.p,
                                    A.dimN, A.T0, A.R, self);
  }
}

}  // namespace

int spectrum_gpu(Setup& s, Error& err) {
  PeriodicGreen G(s.L);
  int U[3], K[3];
  for (int a = 0; a < 3; ++a) {
    U[a] = s.periodic[a] ? s.dims[a] / 2 + 1 : s.dims[a];   // distinct offsets |d|
    K[a] = s.fft[a] / 2 + 1;                                // distinct wavenumbers |k|
  }
  const int64_t nU = (int64_t)U[0] * U[1] * U[2];
  sm::PgfParams P = G.params();
  DBuf dk;
  int rc;
  if ((rc = dput(dk, G.kflat().data(), G.kflat().size(), err))) return rc;
  P.kvec = dk.as<double>();
  int64_t cap = nU;
  {
    int sh[3] = {U[0], U[1], U[2]};
    for (int a = 0; a < 3; ++a) {
      sh[a] = K[a];
      cap = std::max<int64_t>(cap, (int64_t)sh[0] * sh[1] * sh[2]);
    }
  }
  DBuf cur, nxt;
  if ((rc = dalloc(cur, cap * sizeof(double), err))) return rc;
  if ((rc = dalloc(nxt, cap * sizeof(double), err))) return rc;
  k_pgf_offsets<<<grid_for(nU, 128), 128>>>(P, s.delta[0], s.delta[1], s.delta[2], U[0], U[1], nU, cur.as<double>());
  SG_CK("PGF offsets kernel", cudaGetLastError());
  // even real kernel: FFT = separable cosine sums, sum_d c_d K(d) cos(2 pi d k / F),
  // c_d = 1 at d = 0 and at d = F/2, 2 otherwise (the host set-up's table, to the bit)
  int shape[3] = {U[0], U[1], U[2]};
  for (int a = 0; a < 3; ++a) {
    const int F = s.fft[a];
    std::vector<double> tab((size_t)K[a] * shape[a]);
    for (int k = 0; k < K[a]; ++k)
      for (int d = 0; d < shape[a]; ++d) {
        const double c = (d == 0 || 2 * d == F) ? 1.0 : 2.0;
        tab[(size_t)k * shape[a] + d] = c * std::cos(2.0 * kPi * (double)(((int64_t)d * k) % F) / F);
      }
    DBuf dt;
    if ((rc = dput(dt, tab.data(), tab.size(), err))) return rc;
    int ns[3] = {shape[0], shape[1], shape[2]};
    ns[a] = K[a];
    const int64_t nout = (int64_t)ns[0] * ns[1] * ns[2];
    k_cos_axis<<<grid_for(nout, 128), 128>>>(cur.as<double>(), nxt.as<double>(), dt.as<double>(), shape[0], shape[1],
                                             shape[2], a, K[a], nout);
    SG_CK("cosine transform kernel", cudaGetLastError());
    std::swap(cur.p, nxt.p);
    shape[a] = K[a];
  }
  s.ghat.resize((size_t)K[0] * K[1] * K[2]);
  SG_CK("copy spectrum", cudaMemcpy(s.ghat.data(), cur.p, s.ghat.size() * sizeof(double), cudaMemcpyDeviceToHost));
  return OK;
}

int near_eval_gpu(const Setup& s, const NearPlan& plan, std::vector<double>& out, Error& err) {
  const int64_t Np = s.Np;
  DBuf xyz, tets, bf, lca, pos, pptr, elem, img, dest, dout;
  int rc;
  if ((rc = dput(xyz, s.xyz.data(), s.xyz.size(), err)) || (rc = dput(tets, s.tets.data(), s.tets.size(), err)) ||
      (rc = dput(bf, s.bfaces.data(), s.bfaces.size(), err)) || (rc = dput(lca, s.lca.data(), s.lca.size(), err)) ||
      (rc = dput(pos, s.pos_f.data(), s.pos_f.size(), err)) ||
      (rc = dput(pptr, plan.pptr.data(), plan.pptr.size(), err)) ||
      (rc = dput(elem, plan.elem.data(), plan.elem.size(), err)) ||
      (rc = dput(img, plan.img.data(), plan.img.size(), err)) ||
      (rc = dput(dest, plan.dest.data(), plan.dest.size(), err)) ||
      (rc = dalloc(dout, out.size() * sizeof(double), err)))
    return rc;
  SG_CK("clear", cudaMemset(dout.p, 0, out.size() * sizeof(double)));
  sm::NearArgs A;
  A.xyz = xyz.as<double>();
  A.tets = tets.as<int32_t>();
  A.bfaces = bf.as<int32_t>();
  A.lca = lca.as<int32_t>();
  A.pos_f = pos.as<double>();
  for (int d = 0; d < 3; ++d) A.L[d] = s.periodic[d] ? s.L[d] : 0.0;
  A.T = s.T;
  A.self_tol = 1e-6 * s.mean_edge;
  A.pptr = pptr.as<int64_t>();
  A.elem = elem.as<int64_t>();
  A.img = img.as<int32_t>();
  A.dest = dest.as<int64_t>();
  k_near_rows<<<grid_for(Np, 128), 128>>>(A, Np, dout.as<double>());
  SG_CK("near-element kernel", cudaGetLastError());
  SG_CK("copy near-element values", cudaMemcpy(out.data(), dout.p, out.size() * sizeof(double), cudaMemcpyDeviceToHost));
  return OK;
}

int precorrection_gpu(Setup& s, const std::vector<int32_t>& box, const std::vector<int64_t>& bptr,
                      const std::vector<int32_t>& bl, const std::vector<double>& T0, int R, Error& err) {
  const int64_t Np = s.Np;
  DBuf pos, base, frac, dbox, dbptr, dbl, dT0, dlen, drp, dcol, dval;
  int rc;
  if ((rc = dput(pos, s.pos_f.data(), s.pos_f.size(), err)) || (rc = dput(base, s.base.data(), s.base.size(), err)) ||
      (rc = dput(frac, s.frac.data(), s.frac.size(), err)) || (rc = dput(dbox, box.data(), box.size(), err)) ||
      (rc = dput(dbptr, bptr.data(), bptr.size(), err)) || (rc = dput(dbl, bl.data(), bl.size(), err)) ||
      (rc = dput(dT0, T0.data(), T0.size(), err)) || (rc = dalloc(dlen, (size_t)std::max<int64_t>(Np, 1) * 4, err)))
    return rc;
  PrecorrArgs A;
  A.pos_f = pos.as<double>();
  A.base = base.as<int32_t>();
  A.frac = frac.as<double>();
  A.box = dbox.as<int32_t>();
  A.bptr = dbptr.as<int64_t>();
  A.bl = dbl.as<int32_t>();
  A.T0 = dT0.as<double>();
  A.R = R;
  for (int a = 0; a < 3; ++a) {
    A.dimN[a] = s.dims[a];
    A.per[a] = s.periodic[a] ? 1 : 0;
    A.L[a] = s.L[a];
  }
  A.p = s.p;
  A.nb = s.near_boxes;
  A.Np = Np;
  if (Np > 0) {
    k_precorr_count<<<grid_for(Np, 128), 128>>>(A, dlen.as<int32_t>());
    SG_CK("precorrection count kernel", cudaGetLastError());
  }
  std::vector<int32_t> len(Np);
  if (Np) SG_CK("copy row lengths", cudaMemcpy(len.data(), dlen.p, Np * sizeof(int32_t), cudaMemcpyDeviceToHost));
  std::vector<int64_t> rp(Np + 1, 0);
  int32_t lmax = 0;
  for (int64_t n = 0; n < Np; ++n) {
    rp[n + 1] = rp[n] + len[n];
    lmax = std::max(lmax, len[n]);
  }
  const int64_t nnz = rp[Np];
  if (nnz > 2000000000LL) {
    err = {EINVAL_, "point precorrection has more than 2e9 entries"};
    return EINVAL_;
  }
  int S = 32;
  while (S < lmax) S <<= 1;
  // keys of 4 warps per block in shared memory (fewer warps for very long rows)
  int wpb = 4;
  while (wpb > 1 && (size_t)wpb * S * 8 > 96 * 1024) wpb >>= 1;
  const size_t smem = (size_t)wpb * S * 8;
  if (smem > 200 * 1024) {
    err = {EINVAL_, "GPU set-up: a precorrection row of " + std::to_string(lmax) +
                        " entries exceeds its shared-memory sort; use the host set-up"};
    return EINVAL_;
  }
  if ((rc = dput(drp, rp.data(), rp.size(), err)) || (rc = dalloc(dcol, (size_t)nnz * 4, err)) ||
      (rc = dalloc(dval, (size_t)nnz * 8, err)))
    return rc;
  if (Np > 0) {
    SG_CK("shared-memory size", cudaFuncSetAttribute(k_precorr_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem));
    const int64_t threads = Np * 32;
    const int bs = 32 * wpb;
    k_precorr_fill<<<grid_for(threads, bs), bs, smem>>>(A, drp.as<int64_t>(), S, dcol.as<int32_t>(),
                                                         dval.as<double>());
    SG_CK("precorrection fill kernel", cudaGetLastError());
  }
  s.C.rows = Np;
  s.C.comps = 1;
  s.C.rowptr.resize(Np + 1);
  for (int64_t n = 0; n <= Np; ++n) s.C.rowptr[n] = (int32_t)rp[n];
  s.C.col.resize(nnz);
  s.C.vals.resize(nnz);
  if (nnz) {
    SG_CK("copy precorrection columns", cudaMemcpy(s.C.col.data(), dcol.p, nnz * 4, cudaMemcpyDeviceToHost));
    SG_CK("copy precorrection values", cudaMemcpy(s.C.vals.data(), dval.p, nnz * 8, cudaMemcpyDeviceToHost));
  }
  return OK;
}

}  // namespace pmfem
