// C-ABI of libpmfem (declared in include/pmfem.h).
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pmfem.h"
#include "device.hpp"
#include "internal.hpp"
#include "bloch.hpp"
#include "implicit.hpp"
#include "state.hpp"

using namespace pmfem;

#ifndef PMFEM_NVTX
#define PMFEM_NVTX 1
#endif
#ifndef PMFEM_CHECKS
#define PMFEM_CHECKS 0
#endif


namespace {

thread_local std::string g_create_error;
const double kGammaE = 1.76085963023e11;   // electron gyromagnetic ratio, rad/(s T)

int fail(pmfem_t h, int code, const std::string& msg) {
  if (h) h->err = {code, msg};
  else g_create_error = msg;
  return code;
}

#define PMFEM_CK(h, x)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) return fail(h, ECUDA_, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void prof_hook(void* ctx, int id, int phase, cudaStream_t st) {
  pmfem_t h = (pmfem_t)ctx;
  if (h->ev_next >= h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    h->ev_pool.push_back(e);
  }
  cudaEvent_t e = h->ev_pool[h->ev_next++];
  cudaEventRecord(e, st);
  if (phase == 0) {
    h->open_ev[id] = e;
  } else {
    h->recs.push_back({id, h->open_ev[id], e});
  }
}

void apply_prof(pmfem_t h) {
  ProfHook hk;
  if (h->prof_on) {
    hk.fn = prof_hook;
    hk.ctx = h;
  }
  h->d64.prof = hk;
  h->d32.prof = hk;
  if (h->net) h->net->prof = hk;
}

// Fixed scratch of pmfem_field_noalloc (see the section of that entry point below): one
// file-scope device array, reserved on a device when this library's device code is loaded
// there, and kept until the process exits.
constexpr size_t kNoAllocBytes = 64u << 20;   // 64 MiB of shared scratch per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// In host code g_noalloc_scratch is only a host-side stand-in; the array's device address
// comes from cudaGetSymbolAddress, in the context current now.  Called where the device data
// of a handle are built (a path that may allocate: the lookup can load the module that holds
// the array), so that pmfem_field_noalloc itself only reads the cached address.  A failed
// lookup leaves nullptr and its message; pmfem_field_noalloc then reports it.
void noalloc_lookup(pmfem_t h, std::string* why) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    if (e != cudaSuccess) cudaGetLastError();   // not sticky: clear it for the callers' next check
    *why = std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") + cudaGetErrorString(e);
    p = nullptr;
  }
  h->noalloc_base = p;
}

void free_device(pmfem_t h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  h->d64 = DevOps<double>();
  h->d32 = DevOps<float>();
  h->m = h->mA = h->mB = h->acc = h->mF = h->hin = h->hout = nullptr;
  h->flag = nullptr;
  h->noalloc_base = nullptr;
  h->imp_vec.clear();
  h->imp_pinv = h->imp_c = h->imp_red = nullptr;
  h->imp_prec = -1;
  h->bloch_spec = nullptr;
  h->bloch_buf[0] = h->bloch_buf[1] = h->bloch_buf[2] = nullptr;
  h->bloch_prec = -1;
  h->dev_ready = false;
  h->dev_prec = -1;
}

// Test hook (pmfem_debug_fail_alloc): when >= 0, the number of device allocations still
// allowed before dalloc reports ENOMEM without calling the allocator.
std::atomic<int> g_fail_after{-1};

int dalloc(pmfem_t h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  for (int left = g_fail_after.load(); left >= 0; left = g_fail_after.load()) {
    if (left == 0) return fail(h, ENOMEM_, "device allocation refused by pmfem_debug_fail_alloc");
    if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(h, e == cudaErrorMemoryAllocation ? ENOMEM_ : ECUDA_,
                std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  return OK;
}

template <typename X>
int upload(pmfem_t h, const X* src, size_t n, const X** out) {
  void* p;
  int rc = dalloc(h, &p, n * sizeof(X));
  if (rc) return rc;
  if (n) PMFEM_CK(h, cudaMemcpy(p, src, n * sizeof(X), cudaMemcpyHostToDevice));
  *out = (const X*)p;
  return OK;
}

template <typename T>
int upload_conv(pmfem_t h, const double* src, size_t n, size_t stride, size_t off, double scale, const T** out) {
  std::vector<T> tmp(n);
  for (size_t i = 0; i < n; ++i) tmp[i] = (T)(src[i * stride + off] * scale);
  return upload(h, tmp.data(), n, out);
}

// Nearest bfloat16 (ties to even) of an FP64 value, without double rounding: the value is
// first rounded to FP32 by rounding to odd (truncate toward zero, then set the last bit if
// anything was cut off; Boldo and Melquiond, IEEE Trans. Computers 57(4), 2008), which keeps
// enough of the discarded part for the final round-to-nearest-even at 8 significant bits.
uint16_t bf16_round(double v) {
  if (std::isnan(v)) return 0x7FC0;
  float f = (float)v;
  if (std::isinf(f)) {                       // beyond FP32: beyond bfloat16 as well
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
  }
  if (std::fabs((double)f) > std::fabs(v)) f = std::nextafter(f, 0.0f);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((double)f != v) u |= 1u;
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

int upload_bf16(pmfem_t h, const double* src, size_t n, const bf16_t** out) {
  std::vector<bf16_t> tmp(n);
  for (size_t i = 0; i < n; ++i) tmp[i].bits = bf16_round(src[i]);
  return upload(h, tmp.data(), n, out);
}

template <typename T>
int upload_sell(pmfem_t h, const SellMatrix& M, DevSell<T>& D, unsigned bf_comps = 0) {
  int rc;
  D.rows = M.rows;
  D.col16 = M.col16;
  bool identity = true;
  for (int64_t t = 0; t < M.rows && identity; ++t) identity = M.map[t] == t;
  if (!identity && (rc = upload(h, M.map.data(), M.map.size(), &D.map))) return rc;
  if ((rc = upload(h, M.len.data(), M.len.size(), &D.len))) return rc;
  if ((rc = upload(h, M.base.data(), M.base.size(), &D.base))) return rc;
  // vector loads of a lane's step (up to 32 bytes) need chunk offsets in whole steps
  for (int64_t o : M.off)
    if (o % M.vw) return fail(h, ESTATE_, "internal: SELL chunk offset not a multiple of the vector width");
  if ((rc = upload(h, M.off.data(), M.off.size(), &D.off))) return rc;
  if (M.col16) {
    const int16_t* p16;
    if ((rc = upload(h, M.d16.data(), M.d16.size(), &p16))) return rc;
    D.delta = p16;
  } else {
    const int32_t* p32;
    if ((rc = upload(h, M.d32.data(), M.d32.size(), &p32))) return rc;
    D.delta = p32;
  }
  const int64_t P = M.padded();
  for (int c = 0; c < M.comps; ++c) {
    if (sizeof(T) == 4 && (bf_comps >> c) & 1u) {
      if ((rc = upload_bf16(h, M.val.data() + (size_t)c * P, P, &D.bval[c]))) return rc;
    } else if ((rc = upload_conv<T>(h, M.val.data() + (size_t)c * P, P, 1, 0, 1.0, &D.val[c]))) {
      return rc;
    }
  }
  return OK;
}

template <typename T>
int build_device(pmfem_t h, DevOps<T>& d) {
  using C2 = typename Vec2<T>::type;
  const Setup& s = h->s;
  Layout L;
  {
    Error err;
    int rc = build_layout(s, L, err);
    if (rc) return fail(h, rc, err.msg);
  }
  int rc;
  d.Np = s.Np;
  d.nnz = (int64_t)L.col.size();
  d.nnzC = (int64_t)L.cval.size();
  d.nnzX = L.Ex.nnz();
  d.p = s.p;
  d.nb = s.near_boxes;
  d.TY = L.TY;
  d.TZ = L.TZ;
  d.pl = L.pl;
  d.pr = L.pr;
  for (int a = 0; a < 3; ++a) {
    d.dims[a] = s.dims[a];
    d.fft[a] = s.fft[a];
    d.periodic[a] = s.periodic[a];
  }
  if ((rc = upload(h, L.perm.data(), L.perm.size(), &d.perm))) return rc;
  if (!s.tet_grain.empty()) {
    // volume share of every grain at every unknown (lumped nodal quadrature), internal order
    const int G = (int)(s.grain_tab.size() / kGrainTab);
    std::vector<std::vector<std::pair<int32_t, double>>> gw(s.Np);
    for (int64_t e = 0; e < s.T; ++e) {
      double X[4][3], gr[4][3];
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) X[a][c] = s.xyz[3 * (int64_t)s.tets[4 * e + a] + c];
      const double q = 0.25 * tet_grads(X, gr);
      for (int a = 0; a < 4; ++a) {
        auto& v = gw[s.lca[s.tets[4 * e + a]]];
        bool found = false;
        for (auto& x : v)
          if (x.first == s.tet_grain[e]) {
            x.second += q;
            found = true;
          }
        if (!found) v.push_back({s.tet_grain[e], q});
      }
    }
    std::vector<int32_t> ptr(s.Np + 1, 0), grain;
    std::vector<double> w;
    for (int64_t i = 0; i < s.Np; ++i) {
      const int32_t uo = L.perm[i];
      double tot = 0;
      for (auto& x : gw[uo]) tot += x.second;
      for (auto& x : gw[uo]) {
        grain.push_back(x.first);
        w.push_back(x.second / tot);
      }
      ptr[i + 1] = (int32_t)grain.size();
    }
    (void)G;
    if ((rc = upload(h, ptr.data(), ptr.size(), &d.loc.ptr))) return rc;
    if ((rc = upload(h, grain.data(), grain.size(), &d.loc.grain))) return rc;
    if ((rc = upload_conv<T>(h, w.data(), w.size(), 1, 0, 1.0, &d.loc.w))) return rc;
    if ((rc = upload_conv<T>(h, s.grain_tab.data(), s.grain_tab.size(), 1, 0, 1.0, &d.loc.tab))) return rc;
  }
  // BF16-split: component masks of the operators stored in bfloat16 (adjacency components
  // 0-2 W^q, 3-5 E, 6-8 gradient, 9 exchange)
  const int bo = (sizeof(T) == 4 && h->prec == PMFEM_BF16SPLIT) ? h->bf16_ops : 0;
  const unsigned adj_bf = ((bo & PMFEM_BF16_CHARGES) ? 0x3Fu : 0u) | ((bo & PMFEM_BF16_GRADIENT) ? 0x1C0u : 0u) |
                          ((bo & PMFEM_BF16_EXCHANGE) ? 0x200u : 0u);
  if ((rc = upload_sell(h, L.adj, d.adj, adj_bf))) return rc;
  if ((rc = upload_sell(h, L.cor, d.cor, (bo & PMFEM_BF16_PRECORRECTION) ? 1u : 0u))) return rc;
  if ((rc = upload_sell(h, L.pro, d.pro, (bo & PMFEM_BF16_PROJECTION) ? 1u : 0u))) return rc;
  const SellMatrix* ms[3] = {&L.adj, &L.cor, &L.pro};
  for (int k = 0; k < 3; ++k) {
    int64_t nnz = 0;
    for (int32_t v : ms[k]->len) nnz += v;
    h->dev_info[3 * k] = nnz;
    h->dev_info[3 * k + 1] = ms[k]->padded();
    h->dev_info[3 * k + 2] = ms[k]->col16 ? 16 : 32;
  }
  h->dev_info[9] = (int64_t)L.xnode.size();
  h->dev_info[10] = L.TY;
  h->dev_info[11] = L.TZ;
  h->dev_info[12] = L.pro.rows;

  d.nx_exc = (int64_t)L.xnode.size();
  if ((rc = upload(h, L.xnode.data(), L.xnode.size(), &d.xnode))) return rc;
  if ((rc = upload(h, L.xgrid.data(), L.xgrid.size(), &d.xgrid))) return rc;
  if ((rc = upload_conv<T>(h, L.xw.data(), L.xw.size(), 1, 0, 1.0, &d.xw))) return rc;
  if ((rc = upload(h, L.Ex.rowptr.data(), L.Ex.rowptr.size(), &d.rowptrX))) return rc;
  if ((rc = upload(h, L.Ex.col.data(), L.Ex.col.size(), &d.colX))) return rc;
  if ((rc = upload_conv<T>(h, L.Ex.vals.data(), L.Ex.vals.size(), 1, 0, 1.0, &d.valX))) return rc;
  if ((rc = upload(h, L.base.data(), L.base.size(), &d.base))) return rc;
  if ((rc = upload_conv<T>(h, L.frac.data(), L.frac.size(), 1, 0, 1.0, &d.frac))) return rc;
  const double scale = 1.0 / ((double)s.fft[0] * s.fft[1] * s.fft[2]);
  if ((rc = upload_conv<T>(h, s.ghat.data(), s.ghat.size(), 1, 0, scale, &d.ghat))) return rc;
  for (int a = 0; a < 3; ++a) {
    const int F = s.fft[a];
    std::vector<C2> tw(F);
    for (int j = 0; j < F; ++j) {
      double ang = 2.0 * kPi * j / F;
      tw[j].x = (T)std::cos(ang);
      tw[j].y = (T)(-std::sin(ang));
    }
    if ((rc = upload(h, tw.data(), tw.size(), &d.tw[a]))) return rc;
  }
  void* p;
  const int64_t ngrid = (int64_t)s.dims[0] * s.dims[1] * s.dims[2];
  const int64_t ncb = (int64_t)(s.fft[0] / 2 + 1) * s.fft[1] * s.fft[2];
  if ((rc = dalloc(h, &p, s.Np * sizeof(T)))) return rc;
  d.q = (T*)p;
  if ((rc = dalloc(h, &p, s.Np * sizeof(T)))) return rc;
  d.e = (T*)p;
  if ((rc = dalloc(h, &p, ngrid * sizeof(T)))) return rc;
  d.grid = (T*)p;
  if ((rc = dalloc(h, &p, ncb * sizeof(C2)))) return rc;
  d.cbuf = (C2*)p;
  const size_t sv = (size_t)s.Np * sizeof(V4<T>);
  const size_t su = 3 * (size_t)s.Np * sizeof(T);
  if ((rc = dalloc(h, &h->m, sv))) return rc;
  if ((rc = dalloc(h, &h->mA, sv))) return rc;
  if ((rc = dalloc(h, &h->mB, sv))) return rc;
  if ((rc = dalloc(h, &h->acc, sv))) return rc;
  if ((rc = dalloc(h, &h->mF, sv))) return rc;
  if ((rc = dalloc(h, &h->hin, su))) return rc;
  if ((rc = dalloc(h, &h->hout, su))) return rc;
  if ((rc = dalloc(h, &p, sizeof(int)))) return rc;
  h->flag = (int*)p;
  d.flag = h->flag;
  PMFEM_CK(h, cudaMemset(h->flag, 0, sizeof(int)));
  PMFEM_CK(h, cudaMemset(h->m, 0, sv));
  if (PMFEM_CHECKS) {
    // bounds of every stored index, checked on the device before any kernel uses them;
    // a failure is reported by the next pmfem_sync (EINVAL)
    launch_layout_checks(d, h->stream);
    PMFEM_CK(h, cudaStreamSynchronize(h->stream));
  }
  return OK;
}

int ensure_device(pmfem_t h) {
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity before using the GPU");
  if (h->dev_ready && h->dev_prec == h->prec) return OK;
  free_device(h);
  // a blocking stream: work on it is ordered with the legacy default stream (handle 0)
  if (!h->stream) PMFEM_CK(h, cudaStreamCreate(&h->stream));
  if (!h->side) PMFEM_CK(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  if (!h->ev_fork) PMFEM_CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  if (!h->ev_join) PMFEM_CK(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  const auto t0 = std::chrono::steady_clock::now();
  int rc = (h->prec == PMFEM_FP64) ? build_device(h, h->d64) : build_device(h, h->d32);
  if (rc) {
    free_device(h);
    return rc;
  }
  h->s.t_stage[6] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  h->dev_prec = h->prec;
  h->dev_ready = true;
  noalloc_lookup(h, &h->noalloc_why);
  apply_prof(h);
  return OK;
}

// PMFEM_OVERLAP 1: in FP32 and BF16-split, the precorrection (which needs only q, m and e) runs
// on the handle's side stream, ordered only after the charges, while the projection and the FFT
// produce the grid potential on st (each of these kernels fills the GPU, so the block scheduler
// overlaps them at kernel boundaries); the stencil of that potential is then added in a second,
// light pass (measured on the 1M-node wire: 644 -> 620 us per evaluation in FP32, 559 -> 532 in
// BF16-split).  FP64 keeps
// the fused kernel: its stencil alone takes 367 us on GB300's narrow FP64 units, work that the
// fused kernel hides under the precorrection's memory latency.  0: fused everywhere.  With
// per-launch timing on, the passes run in order on st, so that each launch is timed alone.
#ifndef PMFEM_OVERLAP
#define PMFEM_OVERLAP 1
#endif
// NVTX ranges around the stages of an evaluation (host-side enqueue; header-only NVTX 3, a no-op
// unless a tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) {
    if (PMFEM_NVTX) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (PMFEM_NVTX) nvtxRangePop();
  }
};

template <typename T>
void enqueue_eval(pmfem_t h, DevOps<T>& d, const V4<T>* m, T* H, int comps, const RkArgs& rk, cudaStream_t st) {
  NvtxRange all("pmfem field evaluation");
  if (comps & PMFEM_MS) {
    NvtxRange ms("pmfem magnetostatic: charges, precorrection, projection, FFT, stencil");
    launch_charges(d, m, st);
    if (PMFEM_OVERLAP && sizeof(T) == 4) {
      const bool fork = !h->prof_on && h->side && h->ev_fork && h->ev_join;
      cudaStream_t s2 = fork ? h->side : st;
      if (fork) {
        cudaEventRecord(h->ev_fork, st);
        cudaStreamWaitEvent(s2, h->ev_fork, 0);
      }
      launch_precorr(d, m, s2);
      if (fork) cudaEventRecord(h->ev_join, s2);
      launch_anterp(d, st);
      launch_fft_conv(d, st);
      launch_stencil(d, m, st);     // adds into the potential lane beside the precorrection
      if (fork) cudaStreamWaitEvent(st, h->ev_join, 0);
    } else {
      launch_anterp(d, st);
      launch_fft_conv(d, st);
      launch_interp(d, m, st);
    }
  }
  NvtxRange fr("pmfem gradient + exchange + local terms");
  launch_field(d, m, H, comps, h->hap[0], h->hap[1], h->hap[2], rk, st);
}

int check_launch(pmfem_t h) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, ECUDA_, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  return OK;
}

template <typename T>
int run_llg(pmfem_t h, DevOps<T>& d, double dt, int nsteps, cudaStream_t st) {
  const double gam = kMu0 * kGammaE / (1.0 + h->s.alpha * h->s.alpha);
  V4<T>* m = (V4<T>*)h->m;
  V4<T>* A = (V4<T>*)h->mA;
  V4<T>* B = (V4<T>*)h->mB;
  for (int n = 0; n < nsteps; ++n) {
    RkArgs rk;
    rk.m0 = m;
    rk.acc = h->acc;
    rk.gam = gam;
    rk.alpha = h->s.alpha;
    rk.mode = 1;
    rk.cdt = 0.5 * dt, rk.bw = 1.0, rk.acc_init = 1, rk.mnext = A;
    enqueue_eval(h, d, (const V4<T>*)m, (T*)nullptr, PMFEM_ALL, rk, st);
    rk.cdt = 0.5 * dt, rk.bw = 2.0, rk.acc_init = 0, rk.mnext = B;
    enqueue_eval(h, d, (const V4<T>*)A, (T*)nullptr, PMFEM_ALL, rk, st);
    rk.cdt = dt, rk.bw = 2.0, rk.acc_init = 0, rk.mnext = A;
    enqueue_eval(h, d, (const V4<T>*)B, (T*)nullptr, PMFEM_ALL, rk, st);
    rk.mode = 2;
    rk.dt6 = dt / 6.0;
    enqueue_eval(h, d, (const V4<T>*)A, (T*)nullptr, PMFEM_ALL, rk, st);
    int rc = check_launch(h);
    if (rc) return rc;
  }
  return OK;
}

// ------------------------------------------------------------------------------------
// Implicit midpoint LLG steps with Newton-GMRES (kernels and formulas in implicit.cu).
// The vectors of a step live in the C-ABI order; every field evaluation goes through the
// handle's own path (permute in, the evaluation of pmfem_field), with the applied field for
// the residual and without it for the Jacobian's products (the field's linear part).
// ------------------------------------------------------------------------------------
struct ImpOpts {
  double newton_tol, krylov_tol;
  int restart, max_newton, max_krylov;
};

template <typename T>
int run_implicit(pmfem_t h, DevOps<T>& d, double dt, int nsteps, const ImpOpts& o, int64_t stats[4],
                 cudaStream_t st) {
  const int64_t n = d.Np, len = 3 * n;
  const int k = o.restart;
  const double g = kMu0 * kGammaE / (1.0 + h->s.alpha * h->s.alpha), alpha = h->s.alpha;
  // work vectors (device, allocated with the handle's device data; a longer cycle adds more)
  const int nvec = 9 + (k + 1);
  if ((int)h->imp_vec.size() < nvec || h->imp_prec != h->dev_prec) {
    h->imp_vec.clear();
    for (int i = 0; i < nvec; ++i) {
      void* p;
      int rc = dalloc(h, &p, (size_t)len * sizeof(T));
      if (rc) return rc;
      h->imp_vec.push_back(p);
    }
    void* p;
    int rc;
    if ((rc = dalloc(h, &p, (size_t)9 * n * sizeof(T)))) return rc;
    h->imp_pinv = p;
    if ((rc = dalloc(h, &p, (size_t)std::max<int64_t>(n, 1) * sizeof(T)))) return rc;
    h->imp_c = p;
    if ((rc = dalloc(h, &p, (size_t)(kImpBlocks + 3) * (kMaxKrylov + 1) * sizeof(double)))) return rc;
    h->imp_red = p;
    h->imp_prec = h->dev_prec;
    // the exchange operator's own coefficient of every unknown (preconditioner blocks)
    std::vector<T> c(n, (T)0);
    for (int64_t u = 0; u < n; ++u)
      for (int32_t q = h->s.rowptr[u]; q < h->s.rowptr[u + 1]; ++q)
        if (h->s.col[q] == u) c[u] = (T)h->s.Kp[q];
    PMFEM_CK(h, cudaMemcpy(h->imp_c, c.data(), n * sizeof(T), cudaMemcpyHostToDevice));
  }
  T* m0 = (T*)h->imp_vec[0];
  T* y = (T*)h->imp_vec[1];
  T* mb = (T*)h->imp_vec[2];
  T* Hb = (T*)h->imp_vec[3];
  T* R = (T*)h->imp_vec[4];
  T* x = (T*)h->imp_vec[5];
  T* z = (T*)h->imp_vec[6];
  T* w = (T*)h->imp_vec[7];
  T* Av = (T*)h->imp_vec[8];
  T** V = (T**)&h->imp_vec[9];
  T* Pinv = (T*)h->imp_pinv;
  const T* cdiag = (const T*)h->imp_c;
  double* red = (double*)h->imp_red;                         // partial sums, then results
  double* dres = red + (size_t)kImpBlocks * (kMaxKrylov + 1);
  // Arnoldi step results on the device: both Gram-Schmidt passes' coefficients and |w|^2
  constexpr int K1 = kMaxKrylov + 1;
  double* dA = dres + K1;
  double* dB = dres + 2 * K1;
  double* dC = dB + kMaxKrylov;   // (a cycle has at most kMaxKrylov columns: dB[0 .. j], j < kMaxKrylov)
  const int nblk = (int)std::min<int64_t>(kImpBlocks, std::max<int64_t>(1, (len + 255) / 256));
  RkArgs none;
  auto eval = [&](const T* xin, T* H, int comps) {
    launch_perm_in(d, xin, (V4<T>*)h->mF, st);
    enqueue_eval(h, d, (const V4<T>*)h->mF, H, comps, none, st);
    ++stats[2];
  };
  auto dots = [&](int cnt, T* const* vs, const T* wv, double* out) -> int {
    VecList<T> L;
    for (int j = 0; j < cnt; ++j) L.p[j] = vs[j];
    imp_multidot(len, L, cnt, wv, red, nblk, dres, st);
    PMFEM_CK(h, cudaMemcpyAsync(out, dres, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
    PMFEM_CK(h, cudaStreamSynchronize(st));
    return OK;
  };
  // wv = a wv + sum coef_j vs_j
  auto combine = [&](int cnt, T* const* vs, const double* coef, double a, T* wv) -> int {
    VecList<T> L;
    for (int j = 0; j < cnt; ++j) L.p[j] = vs[j];
    PMFEM_CK(h, cudaMemcpyAsync(dres, coef, cnt * sizeof(double), cudaMemcpyHostToDevice, st));
    imp_combine(len, L, cnt, dres, 1.0, a, wv, st);
    PMFEM_CK(h, cudaStreamSynchronize(st));   // coef is a host array of the caller
    return OK;
  };
  auto Jv = [&](T* v, T* out) {   // out = J v
    eval(v, Av, PMFEM_EX | PMFEM_MS);
    imp_jvp(n, (const T*)mb, (const T*)Hb, (const T*)Av, (const T*)v, dt, g, alpha, out, st);
  };
  // w = J z, the product of every Arnoldi step (fixed buffers), captured once per call as a CUDA
  // graph (the evaluation's launches and its second-stream fork replayed in one launch); the
  // eager launches run instead while per-launch timing is on
  struct GraphGuard {
    cudaGraphExec_t g = nullptr;
    ~GraphGuard() {
      if (g) cudaGraphExecDestroy(g);
    }
  } jvz;
  if (!h->prof_on) {
    cudaStream_t cs;
    PMFEM_CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch_perm_in(d, (const T*)z, (V4<T>*)h->mF, cs);
      enqueue_eval(h, d, (const V4<T>*)h->mF, Av, PMFEM_EX | PMFEM_MS, none, cs);
      imp_jvp(n, (const T*)mb, (const T*)Hb, (const T*)Av, (const T*)z, dt, g, alpha, w, cs);
      e = cudaStreamEndCapture(cs, &gr);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&jvz.g, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(h, ECUDA_, std::string("implicit step: capture of J z failed: ") + cudaGetErrorString(e));
  }
  auto Jz = [&]() -> int {   // w = J z
    if (!jvz.g) {
      Jv(z, w);
      return OK;
    }
    PMFEM_CK(h, cudaGraphLaunch(jvz.g, st));
    ++stats[2];
    return OK;
  };
  double hres[2 * K1];
  int rc;
  launch_perm_out(d, (const V4<T>*)h->m, m0, st);
  for (int step = 0; step < nsteps; ++step) {
    PMFEM_CK(h, cudaMemcpyAsync(y, m0, len * sizeof(T), cudaMemcpyDeviceToDevice, st));
    bool conv = false;
    for (int it = 0; it < o.max_newton && !conv; ++it) {
      imp_mid(n, (const T*)m0, (const T*)y, mb, st);
      eval(mb, Hb, PMFEM_ALL);
      imp_residual(n, (const T*)m0, (const T*)y, (const T*)mb, (const T*)Hb, dt, g, alpha, R, st);
      imp_blocks(n, (const T*)mb, (const T*)Hb, cdiag, dt, g, alpha, Pinv, st);
      ++stats[0];
      // GMRES on J x = -R, x0 = 0, right-preconditioned by the blocks, restarted every k
      double one = 1.0, mone = -1.0, zero = 0.0;
      (void)zero;
      PMFEM_CK(h, cudaMemsetAsync(x, 0, len * sizeof(T), st));
      double b2;
      if ((rc = dots(1, &R, R, &b2))) return rc;
      const double bnorm = std::sqrt(b2);
      double beta = bnorm;
      // r = -R into V[0] (scaled below)
      if ((rc = combine(1, &R, &mone, 0.0, V[0]))) return rc;
      int kits = 0;
      while (beta > o.krylov_tol * bnorm && beta > 0 && kits < o.max_krylov) {
        double inv = 1.0 / beta;
        if ((rc = combine(1, &V[0], &inv, 0.0, V[0]))) return rc;
        std::vector<double> Hm((size_t)(k + 1) * k, 0.0), cs(k), sn(k), gv(k + 1, 0.0);
        gv[0] = beta;
        int j = 0;
        for (; j < k && kits < o.max_krylov; ++j) {
          imp_apply_blocks(n, (const T*)Pinv, (const T*)V[j], z, st);
          if ((rc = Jz())) return rc;
          ++kits;
          ++stats[1];
          // classical Gram-Schmidt twice and the normalisation, with the coefficients kept on
          // the device between the passes; one copy back per step for the Hessenberg column
          VecList<T> L;
          for (int i = 0; i <= j; ++i) L.p[i] = V[i];
          imp_multidot(len, L, j + 1, (const T*)w, red, nblk, dA, st);
          imp_combine(len, L, j + 1, dA, -1.0, 1.0, w, st);
          imp_multidot(len, L, j + 1, (const T*)w, red, nblk, dB, st);
          imp_combine(len, L, j + 1, dB, -1.0, 1.0, w, st);
          VecList<T> Lw;
          Lw.p[0] = w;
          imp_multidot(len, Lw, 1, (const T*)w, red, nblk, dC, st);
          imp_scale_invnorm(len, (const T*)w, dC, V[j + 1], st);
          PMFEM_CK(h, cudaMemcpyAsync(hres, dA, 2 * K1 * sizeof(double), cudaMemcpyDeviceToHost, st));
          PMFEM_CK(h, cudaStreamSynchronize(st));
          for (int i = 0; i <= j; ++i) Hm[(size_t)i * k + j] = hres[i] + hres[K1 + i];
          const double wn = std::sqrt(std::max(hres[K1 + kMaxKrylov], 0.0));
          Hm[(size_t)(j + 1) * k + j] = wn;
          // Givens rotations of column j
          for (int i = 0; i < j; ++i) {
            const double a = Hm[(size_t)i * k + j], b = Hm[(size_t)(i + 1) * k + j];
            Hm[(size_t)i * k + j] = cs[i] * a + sn[i] * b;
            Hm[(size_t)(i + 1) * k + j] = -sn[i] * a + cs[i] * b;
          }
          const double a = Hm[(size_t)j * k + j], b = Hm[(size_t)(j + 1) * k + j];
          const double r = std::hypot(a, b);
          cs[j] = r > 0 ? a / r : 1.0;
          sn[j] = r > 0 ? b / r : 0.0;
          Hm[(size_t)j * k + j] = r;
          Hm[(size_t)(j + 1) * k + j] = 0.0;
          gv[j + 1] = -sn[j] * gv[j];
          gv[j] = cs[j] * gv[j];
          beta = std::fabs(gv[j + 1]);
          if (beta <= o.krylov_tol * bnorm || wn == 0) {
            ++j;
            break;
          }
        }
        // x += P^-1 (V_{0..j-1} yv), yv from the triangular system
        std::vector<double> yv(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
          double s2 = gv[i];
          for (int l = i + 1; l < j; ++l) s2 -= Hm[(size_t)i * k + l] * yv[l];
          yv[i] = Hm[(size_t)i * k + i] != 0 ? s2 / Hm[(size_t)i * k + i] : 0.0;
        }
        if ((rc = combine(j, V, yv.data(), 0.0, w))) return rc;
        imp_apply_blocks(n, (const T*)Pinv, (const T*)w, z, st);
        if ((rc = combine(1, &z, &one, 1.0, x))) return rc;
        if (beta <= o.krylov_tol * bnorm || kits >= o.max_krylov) break;
        // restart: r = -R - J x
        Jv(x, w);
        T* pair[2] = {R, w};
        double cf[2] = {-1.0, -1.0};
        if ((rc = combine(2, pair, cf, 0.0, V[0]))) return rc;
        double r2;
        if ((rc = dots(1, &V[0], V[0], &r2))) return rc;
        beta = std::sqrt(r2);
      }
      // y += x; converged when |x| <= newton_tol |y|
      if ((rc = combine(1, &x, &one, 1.0, y))) return rc;
      double xx, yy;
      if ((rc = dots(1, &x, x, &xx))) return rc;
      if ((rc = dots(1, &y, y, &yy))) return rc;
      if (!std::isfinite(xx) || !std::isfinite(yy))
        return fail(h, ENONFINITE_, "implicit step: non-finite Newton iterate");
      conv = std::sqrt(xx) <= o.newton_tol * std::sqrt(yy);
    }
    if (!conv) {
      return fail(h, ENOCONV_, "implicit step " + std::to_string(step) + ": Newton did not converge in " +
                                   std::to_string(o.max_newton) + " iterations (dt too large for this state?)");
    }
    PMFEM_CK(h, cudaMemcpyAsync(m0, y, len * sizeof(T), cudaMemcpyDeviceToDevice, st));
    launch_perm_in(d, (const T*)m0, (V4<T>*)h->m, st);
    ++stats[3];
  }
  return check_launch(h);
}

// RK4 steps with the surrogate: stage 1 runs the full P-AIM and keeps its grid charges Q1
// and potential U1; stages 2-4 take U = U1 + net(Q - Q1) instead of the FFT convolution,
// except on every sur_every-th step, where they run the full P-AIM and the network's
// potential is measured against it.
int run_llg_sur(pmfem_t h, DevOps<float>& d, double dt, int nsteps, cudaStream_t st) {
  SurrogateNet& n = *h->net;
  const double gam = kMu0 * kGammaE / (1.0 + h->s.alpha * h->s.alpha);
  V4<float>* m = (V4<float>*)h->m;
  V4<float>* A = (V4<float>*)h->mA;
  V4<float>* B = (V4<float>*)h->mB;
  const size_t gb = (size_t)n.V * sizeof(float);
  for (int k = 0; k < nsteps; ++k) {
    const bool judge = (h->sur_step % h->sur_every) == 0;
    RkArgs rk;
    rk.m0 = m;
    rk.acc = h->acc;
    rk.gam = gam;
    rk.alpha = h->s.alpha;
    const V4<float>* in[4] = {m, A, B, A};
    for (int s = 0; s < 4; ++s) {
      rk.mode = s < 3 ? 1 : 2;
      rk.cdt = s < 2 ? 0.5 * dt : dt;
      rk.bw = s == 0 ? 1.0 : 2.0;
      rk.acc_init = s == 0 ? 1 : 0;
      rk.mnext = s == 0 ? (void*)A : s == 1 ? (void*)B : (void*)A;
      rk.dt6 = dt / 6.0;
      launch_charges(d, in[s], st);
      launch_anterp(d, st);
      if (s == 0) {
        PMFEM_CK(h, cudaMemcpyAsync(n.Q1, d.grid, gb, cudaMemcpyDeviceToDevice, st));
        launch_fft_conv(d, st);
        PMFEM_CK(h, cudaMemcpyAsync(n.U1, d.grid, gb, cudaMemcpyDeviceToDevice, st));
      } else if (judge) {
        PMFEM_CK(h, cudaMemcpyAsync(n.gA, d.grid, gb, cudaMemcpyDeviceToDevice, st));
        launch_fft_conv(d, st);
        net_judge(n, n.gA, d.grid, st);
        ++h->sur_judged;
      } else {
        net_increment(n, d.grid, st);
        ++h->sur_evals;
      }
      launch_interp(d, in[s], st);
      launch_field(d, in[s], (float*)nullptr, PMFEM_ALL, h->hap[0], h->hap[1], h->hap[2], rk, st);
    }
    ++h->sur_step;
    int rc = check_launch(h);
    if (rc) return rc;
  }
  return OK;
}

size_t elem_size(pmfem_t h) { return h->prec == PMFEM_FP64 ? sizeof(double) : sizeof(float); }

}  // namespace

extern "C" {

const char* pmfem_version(void) { return "pmfem 0.1 (sm_103a)"; }

const char* pmfem_last_error(pmfem_t h) {
  if (!h) return g_create_error.c_str();
  return h->err.msg.c_str();
}

int pmfem_create_mesh(pmfem_t* out, const double* xyz, int64_t N, const int32_t* tets, int64_t T, double Ms,
                      double A, double alpha) {
  if (!out) return fail(nullptr, EINVAL_, "out is NULL");
  *out = nullptr;
  if (!xyz || !tets || N < 4 || T < 1) return fail(nullptr, EINVAL_, "need xyz, tets, N >= 4 and T >= 1");
  if (!(Ms > 0) || !(A >= 0) || !(alpha >= 0) || !std::isfinite(Ms) || !std::isfinite(A) || !std::isfinite(alpha))
    return fail(nullptr, EINVAL_, "need Ms > 0, A >= 0, alpha >= 0 (finite)");
  pmfem_state* h = nullptr;
  try {
    h = new pmfem_state();
    h->s.N = N;
    h->s.T = T;
    h->s.xyz.assign(xyz, xyz + 3 * N);
    h->s.tets.assign(tets, tets + 4 * T);
    h->s.Ms = Ms;
    h->s.A = A;
    h->s.alpha = alpha;
    Error err;
    int rc = setup_validate_mesh(h->s, err);
    if (rc) {
      delete h;
      return fail(nullptr, rc, err.msg);
    }
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(nullptr, ENOMEM_, "host allocation failed");
  }
  *out = h;
  return OK;
}

int pmfem_set_aim(pmfem_t h, int Nx, int Ny, int Nz, int order_p, int near_boxes, double near_elem_factor) {
  if (!h) return EINVAL_;
  int d[3] = {Nx, Ny, Nz};
  for (int a = 0; a < 3; ++a)
    if (d[a] < 0 || (d[a] > 0 && d[a] < 4) || d[a] > 1024) return fail(h, EINVAL_, "grid sizes must be 0 or in [4, 1024]");
  if (order_p != 0 && (order_p < 2 || order_p > 5)) return fail(h, EINVAL_, "order_p must be 0 or in [2, 5]");
  if (near_boxes < 0 || near_boxes > 8) return fail(h, EINVAL_, "near_boxes must be in [0, 8]");
  if (!(near_elem_factor >= 0) || !std::isfinite(near_elem_factor) || near_elem_factor > 10)
    return fail(h, EINVAL_, "near_elem_factor must be in [0, 10]");
  for (int a = 0; a < 3; ++a) h->s.dims_req[a] = d[a];
  h->s.p = order_p ? order_p : 3;
  h->s.near_boxes = near_boxes ? near_boxes : 3;
  h->s.near_elem_factor = near_elem_factor;
  h->s.ready = false;
  free_device(h);
  return OK;
}

int pmfem_set_exchange_per_tet(pmfem_t h, const double* A_tet) {
  if (!h) return EINVAL_;
  if (!A_tet) {
    h->s.A_tet.clear();
    return OK;
  }
  for (int64_t e = 0; e < h->s.T; ++e)
    if (!(A_tet[e] >= 0) || !std::isfinite(A_tet[e])) return fail(h, EINVAL_, "A_tet must be finite and >= 0");
  h->s.A_tet.assign(A_tet, A_tet + h->s.T);
  return OK;
}

int pmfem_set_anisotropy(pmfem_t h, const int32_t* tet_grain, int n_grains, const double* K1, const double* axes,
                         const double* Ku, const double* u) {
  if (!h) return EINVAL_;
  if (!tet_grain) {
    free_device(h);
    h->s.tet_grain.clear();
    h->s.grain_tab.clear();
    return OK;
  }
  if (n_grains <= 0 || !axes || (!K1 && !Ku)) return fail(h, EINVAL_, "need n_grains > 0, axes and K1 or Ku");
  if (Ku && !u) return fail(h, EINVAL_, "Ku needs the uniaxial axes u");
  for (int64_t e = 0; e < h->s.T; ++e)
    if (tet_grain[e] < 0 || tet_grain[e] >= n_grains) return fail(h, EINVAL_, "tet_grain outside [0, n_grains)");
  const double sc = 2.0 / (kMu0 * h->s.Ms);
  std::vector<double> tab((size_t)n_grains * kGrainTab, 0.0);
  for (int g = 0; g < n_grains; ++g) {
    double* P = &tab[(size_t)g * kGrainTab];
    for (int r = 0; r < 3; ++r) {
      const double* a = axes + 9 * g + 3 * r;
      const double nr = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      if (!(std::fabs(nr - 1.0) < 1e-6)) return fail(h, EINVAL_, "grain axes must be unit rows");
      for (int c = 0; c < 3; ++c) P[3 * r + c] = a[c];
    }
    P[9] = K1 ? -sc * K1[g] : 0.0;
    if (Ku) {
      const double* uu = u + 3 * g;
      const double nr = std::sqrt(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
      if (!(nr > 0)) return fail(h, EINVAL_, "uniaxial axes must be non-zero");
      for (int c = 0; c < 3; ++c) P[10 + c] = uu[c] / nr;
      P[13] = sc * Ku[g];
    }
    for (int k = 0; k < kGrainTab; ++k)
      if (!std::isfinite(P[k])) return fail(h, EINVAL_, "non-finite anisotropy parameter");
  }
  free_device(h);   // only an accepted change drops the device data
  h->s.tet_grain.assign(tet_grain, tet_grain + h->s.T);
  h->s.grain_tab.swap(tab);
  return OK;
}

int pmfem_set_setup_device(pmfem_t h, int use_gpu) {
  if (!h) return EINVAL_;
  if (use_gpu != 0 && use_gpu != 1) return fail(h, EINVAL_, "use_gpu must be 0 (host) or 1 (GPU)");
  h->s.setup_gpu = use_gpu == 1;
  return OK;
}

int pmfem_set_layout(pmfem_t h, int tile_y, int tile_z, int sort_window, int col_bits) {
  if (!h) return EINVAL_;
  if (tile_y < 0 || tile_y > 64 || tile_z < 0 || tile_z > 64 || sort_window < 0 || sort_window > 65536)
    return fail(h, EINVAL_, "tile sizes must be in [0, 64] and sort_window in [0, 65536]");
  if (col_bits != 0 && col_bits != 16 && col_bits != 32) return fail(h, EINVAL_, "col_bits must be 0, 16 or 32");
  h->s.tile_y = tile_y;
  h->s.tile_z = tile_z;
  h->s.sort_window = sort_window;
  h->s.col_bits = col_bits;
  free_device(h);
  return OK;
}

int pmfem_set_periodicity(pmfem_t h, double L1, double L2, double L3) {
  if (!h) return EINVAL_;
  double L[3] = {L1, L2, L3};
  for (int a = 0; a < 3; ++a)
    if (!(L[a] >= 0) || !std::isfinite(L[a])) return fail(h, EINVAL_, "periods must be finite and >= 0");
  for (int a = 0; a < 3; ++a) h->s.L[a] = L[a];
  free_device(h);
  try {
    Error err;
    int rc = run_setup(h->s, err);
    if (rc) return fail(h, rc, err.msg);
  } catch (const std::bad_alloc&) {
    return fail(h, ENOMEM_, "host allocation failed during set-up");
  }
  return OK;
}

int pmfem_set_precision(pmfem_t h, int mode) {
  if (!h) return EINVAL_;
  if (mode != PMFEM_FP64 && mode != PMFEM_FP32 && mode != PMFEM_BF16SPLIT)
    return fail(h, EINVAL_, "precision mode must be PMFEM_FP64, PMFEM_FP32 or PMFEM_BF16SPLIT");
  h->prec = mode;
  return OK;
}

int pmfem_set_bf16_operators(pmfem_t h, int mask) {
  if (!h) return EINVAL_;
  const int all = PMFEM_BF16_PRECORRECTION | PMFEM_BF16_PROJECTION | PMFEM_BF16_CHARGES | PMFEM_BF16_GRADIENT |
                  PMFEM_BF16_EXCHANGE;
  if (mask & ~all) return fail(h, EINVAL_, "bf16 operator mask has bits outside the PMFEM_BF16_* flags");
  if (mask != h->bf16_ops && h->dev_prec == PMFEM_BF16SPLIT) free_device(h);   // re-upload at next use
  h->bf16_ops = mask;
  return OK;
}

int pmfem_set_applied_field(pmfem_t h, double Hx, double Hy, double Hz) {
  if (!h) return EINVAL_;
  if (!std::isfinite(Hx) || !std::isfinite(Hy) || !std::isfinite(Hz)) return fail(h, EINVAL_, "applied field not finite");
  h->hap[0] = Hx;
  h->hap[1] = Hy;
  h->hap[2] = Hz;
  if (h->graph) cudaGraphExecDestroy(h->graph);   // the captured step holds the old field
  h->graph = nullptr;
  return OK;
}

int pmfem_num_unknowns(pmfem_t h, int64_t* n) {
  if (!h || !n) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  *n = h->s.Np;
  return OK;
}

int pmfem_lca_map(pmfem_t h, int32_t* out) {
  if (!h || !out) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  std::memcpy(out, h->s.lca.data(), sizeof(int32_t) * h->s.N);
  return OK;
}

int pmfem_field(pmfem_t h, const void* m, void* H, int components, void* stream) {
  if (!h) return EINVAL_;
  if (!m || !H || m == H) return fail(h, EINVAL_, "m and H must be distinct device pointers");
  if (components <= 0 || components > PMFEM_ALL) return fail(h, EINVAL_, "components must be a non-empty PMFEM_EX|MS|AP|AN mask");
  int rc = ensure_device(h);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  RkArgs none;
  if (h->dev_prec == PMFEM_FP64) {
    launch_perm_in(h->d64, (const double*)m, (V4<double>*)h->mF, st);
    enqueue_eval(h, h->d64, (const V4<double>*)h->mF, (double*)H, components, none, st);
  } else {
    launch_perm_in(h->d32, (const float*)m, (V4<float>*)h->mF, st);
    enqueue_eval(h, h->d32, (const V4<float>*)h->mF, (float*)H, components, none, st);
  }
  return check_launch(h);
}

int pmfem_field_host(pmfem_t h, const void* m_host, void* H_host, int components, void* stream) {
  if (!h) return EINVAL_;
  if (!m_host || !H_host) return fail(h, EINVAL_, "NULL host buffer");
  int rc = ensure_device(h);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  const size_t bytes = 3 * (size_t)h->s.Np * elem_size(h);
  PMFEM_CK(h, cudaMemcpyAsync(h->hin, m_host, bytes, cudaMemcpyHostToDevice, st));
  rc = pmfem_field(h, h->hin, h->hout, components, st);
  if (rc) return rc;
  PMFEM_CK(h, cudaMemcpyAsync(H_host, h->hout, bytes, cudaMemcpyDeviceToHost, st));
  PMFEM_CK(h, cudaStreamSynchronize(st));
  return OK;
}

int pmfem_set_m(pmfem_t h, const void* m, void* stream) {
  if (!h || !m) return EINVAL_;
  int rc = ensure_device(h);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (h->dev_prec == PMFEM_FP64) launch_perm_in(h->d64, (const double*)m, (V4<double>*)h->m, st);
  else launch_perm_in(h->d32, (const float*)m, (V4<float>*)h->m, st);
  return check_launch(h);
}

int pmfem_get_m(pmfem_t h, void* m, void* stream) {
  if (!h || !m) return EINVAL_;
  int rc = ensure_device(h);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (h->dev_prec == PMFEM_FP64) launch_perm_out(h->d64, (const V4<double>*)h->m, (double*)m, st);
  else launch_perm_out(h->d32, (const V4<float>*)h->m, (float*)m, st);
  return check_launch(h);
}

int pmfem_llg_step(pmfem_t h, double dt, int nsteps, void* stream) {
  if (!h) return EINVAL_;
  if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return fail(h, EINVAL_, "need dt > 0 and nsteps >= 0");
  int rc = ensure_device(h);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (h->net && h->sur_every > 0 && h->dev_prec != PMFEM_FP64) return run_llg_sur(h, h->d32, dt, nsteps, st);
  if (h->prof_on || nsteps == 0)   // per-launch timing needs the launches themselves
    return h->dev_prec == PMFEM_FP64 ? run_llg(h, h->d64, dt, nsteps, st) : run_llg(h, h->d32, dt, nsteps, st);
  if (!h->graph || h->graph_dt != dt) {
    // capture one step on a private stream, after the caller's work (the capture reads the
    // state buffers by address only); the FFT and interpolation kernels opt into large shared
    // memory first (their scratch outputs are rewritten by the step itself)
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    PMFEM_CK(h, cudaStreamSynchronize(st));
    // (on the scratch input mF, not the state: these launches write the potential lane, which
    // must enter every evaluation of the state at zero)
    if (h->dev_prec == PMFEM_FP64) {
      launch_fft_conv(h->d64, h->stream);
      launch_interp(h->d64, (const V4<double>*)h->mF, h->stream);
      launch_precorr(h->d64, (const V4<double>*)h->mF, h->stream);
    } else {
      launch_fft_conv(h->d32, h->stream);
      launch_interp(h->d32, (const V4<float>*)h->mF, h->stream);
      launch_precorr(h->d32, (const V4<float>*)h->mF, h->stream);
    }
    PMFEM_CK(h, cudaStreamSynchronize(h->stream));
    cudaStream_t cs;
    PMFEM_CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      if (h->dev_prec == PMFEM_FP64) run_llg(h, h->d64, dt, 1, cs);
      else run_llg(h, h->d32, dt, 1, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      h->graph = nullptr;
      return fail(h, ECUDA_, std::string("RK4 step capture failed: ") + cudaGetErrorString(e));
    }
    h->graph_dt = dt;
  }
  for (int k = 0; k < nsteps; ++k) PMFEM_CK(h, cudaGraphLaunch(h->graph, st));
  return OK;
}

int pmfem_llg_step_implicit(pmfem_t h, double dt, int nsteps, const pmfem_implicit_opts* opts, int64_t* stats,
                            void* stream) {
  if (!h) return EINVAL_;
  if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return fail(h, EINVAL_, "need dt > 0 and nsteps >= 0");
  int rc = ensure_device(h);
  if (rc) return rc;
  const bool f64 = h->dev_prec == PMFEM_FP64;
  ImpOpts o;
  o.newton_tol = opts && opts->newton_tol > 0 ? opts->newton_tol : (f64 ? 1e-10 : 1e-5);
  o.krylov_tol = opts && opts->krylov_tol > 0 ? opts->krylov_tol : (f64 ? 1e-8 : 1e-4);
  o.restart = opts && opts->restart > 0 ? opts->restart : 30;
  o.max_newton = opts && opts->max_newton > 0 ? opts->max_newton : 20;
  o.max_krylov = opts && opts->max_krylov > 0 ? opts->max_krylov : 600;
  if (o.restart > kMaxKrylov) return fail(h, EINVAL_, "restart must be at most 64");
  if (!(o.newton_tol < 1) || !(o.krylov_tol < 1)) return fail(h, EINVAL_, "tolerances must be below 1");
  int64_t st4[4] = {0, 0, 0, 0};
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  rc = f64 ? run_implicit(h, h->d64, dt, nsteps, o, st4, st) : run_implicit(h, h->d32, dt, nsteps, o, st4, st);
  if (stats)
    for (int i = 0; i < 4; ++i) stats[i] = st4[i];
  return rc;
}

int pmfem_bloch_spectrum(pmfem_t h, const double* k0, double* out, double* max_imag) {
  if (!h || !k0 || !out) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  Error err;
  {   // k0 checked before any device allocation
    sm::BlochParams P;
    std::vector<double> kv;
    if (int rc = bloch_params(h->s, k0, P, kv, err)) return fail(h, rc, err.msg);
  }
  const int64_t n = (int64_t)h->s.fft[0] * h->s.fft[1] * h->s.fft[2];
  double* d = nullptr;
  PMFEM_CK(h, cudaMalloc(&d, n * sizeof(double)));
  int rc = bloch_spectrum_device(h->s, k0, d, max_imag, err);
  if (!rc) {
    cudaError_t e = cudaMemcpy(out, d, n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      err = {ECUDA_, std::string("copy of the Bloch spectrum: ") + cudaGetErrorString(e)};
      rc = ECUDA_;
    }
  }
  cudaFree(d);
  return rc ? fail(h, rc, err.msg) : OK;
}

int pmfem_bloch_convolve(pmfem_t h, const double* k0, const void* Q, void* U, void* stream) {
  if (!h || !k0 || !Q || !U || Q == U) return fail(h, EINVAL_, "k0, Q and U are required and Q, U distinct");
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  {   // k0 checked before the device data are built
    sm::BlochParams P;
    std::vector<double> kv;
    Error err;
    if (int rc = bloch_params(h->s, k0, P, kv, err)) return fail(h, rc, err.msg);
  }
  int rc = ensure_device(h);
  if (rc) return rc;
  const int64_t n = (int64_t)h->s.fft[0] * h->s.fft[1] * h->s.fft[2];
  const bool f64 = h->dev_prec == PMFEM_FP64;
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  if (!h->bloch_spec || h->bloch_prec != h->dev_prec || h->bloch_k0[0] != k0[0] || h->bloch_k0[1] != k0[1] ||
      h->bloch_k0[2] != k0[2]) {
    if (!h->bloch_spec || h->bloch_prec != h->dev_prec) {
      if ((rc = dalloc(h, &h->bloch_spec, n * es))) return rc;
      if ((rc = dalloc(h, &h->bloch_buf[0], n * 2 * es))) return rc;
    }
    double* d = nullptr;
    PMFEM_CK(h, cudaMalloc(&d, n * sizeof(double)));
    Error err;
    rc = bloch_spectrum_device(h->s, k0, d, nullptr, err);
    if (!rc) {
      if (f64) {
        cudaMemcpy(h->bloch_spec, d, n * sizeof(double), cudaMemcpyDeviceToDevice);
      } else {
        std::vector<double> hs(n);
        std::vector<float> hf(n);
        cudaMemcpy(hs.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < n; ++i) hf[i] = (float)hs[i];
        cudaMemcpy(h->bloch_spec, hf.data(), n * sizeof(float), cudaMemcpyHostToDevice);
      }
    }
    cudaFree(d);
    if (rc) return fail(h, rc, err.msg);
    for (int a = 0; a < 3; ++a) h->bloch_k0[a] = k0[a];
    h->bloch_prec = h->dev_prec;
  }
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (f64) {
    const void* tw[3] = {h->d64.tw[0], h->d64.tw[1], h->d64.tw[2]};
    bloch_convolve_device<double>(h->s, (const double*)h->bloch_spec, Q, U, h->bloch_buf[0], tw, st);
  } else {
    const void* tw[3] = {h->d32.tw[0], h->d32.tw[1], h->d32.tw[2]};
    bloch_convolve_device<float>(h->s, (const float*)h->bloch_spec, Q, U, h->bloch_buf[0], tw, st);
  }
  return check_launch(h);
}

int pmfem_sync(pmfem_t h) {
  if (!h) return EINVAL_;
  if (!h->dev_ready) return OK;
  PMFEM_CK(h, cudaDeviceSynchronize());
  int flag = 0;
  PMFEM_CK(h, cudaMemcpy(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    PMFEM_CK(h, cudaMemset(h->flag, 0, sizeof(int)));
    if (flag & FLAG_LAYOUT) return fail(h, EINVAL_, "device layout check failed (PMFEM_CHECKS build)");
    return fail(h, ENONFINITE_, (flag & FLAG_NONFINITE_IN) ? "non-finite magnetisation input"
                                                          : "non-finite field result");
  }
  return OK;
}

int pmfem_profile(pmfem_t h, int enable) {
  if (!h) return EINVAL_;
  h->prof_on = enable != 0;
  h->recs.clear();
  h->ev_next = 0;
  for (int i = 0; i < KID_COUNT; ++i) {
    h->prof_count[i] = 0;
    h->prof_ms[i] = 0;
  }
  if (h->prof_on && h->ev_pool.size() < 4096) {
    while (h->ev_pool.size() < 4096) {
      cudaEvent_t e;
      PMFEM_CK(h, cudaEventCreate(&e));
      h->ev_pool.push_back(e);
    }
  }
  apply_prof(h);
  return OK;
}

int pmfem_profile_read(pmfem_t h, int64_t* counts, double* total_ms, int n) {
  if (!h || !counts || !total_ms || n <= 0) return EINVAL_;
  PMFEM_CK(h, cudaDeviceSynchronize());
  for (auto& r : h->recs) {
    float ms = 0;
    PMFEM_CK(h, cudaEventElapsedTime(&ms, r.a, r.b));
    h->prof_count[r.id] += 1;
    h->prof_ms[r.id] += ms;
  }
  h->recs.clear();
  h->ev_next = 0;
  for (int i = 0; i < n; ++i) {
    counts[i] = i < KID_COUNT ? h->prof_count[i] : 0;
    total_ms[i] = i < KID_COUNT ? h->prof_ms[i] : 0.0;
  }
  return OK;
}

int pmfem_destroy(pmfem_t h) {
  if (!h) return OK;
  free_device(h);
  if (h->net) {
    net_destroy(*h->net);
    delete h->net;
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return OK;
}

int pmfem_operator_info(pmfem_t h, int which, int64_t* rows, int64_t* nnz, int* comps) {
  if (!h || !rows || !nnz || !comps) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  const Setup& s = h->s;
  *rows = s.Np;
  switch (which) {
    case 0: *nnz = (int64_t)s.col.size(); *comps = 1; break;
    case 1: case 2: case 3: *nnz = (int64_t)s.col.size(); *comps = 3; break;
    case 4: *nnz = s.C.nnz(); *comps = 1; break;
    case 5: *nnz = s.Ex.nnz(); *comps = 3; break;
    default: return fail(h, EINVAL_, "which must be in 0..5");
  }
  return OK;
}

int pmfem_operator_export(pmfem_t h, int which, int32_t* rowptr, int32_t* col, double* vals) {
  int64_t rows, nnz;
  int comps;
  int rc = pmfem_operator_info(h, which, &rows, &nnz, &comps);
  if (rc) return rc;
  if (!rowptr || !col || !vals) return fail(h, EINVAL_, "NULL output");
  const Setup& s = h->s;
  const std::vector<int32_t>& rp = which == 4 ? s.C.rowptr : which == 5 ? s.Ex.rowptr : s.rowptr;
  const std::vector<int32_t>& cl = which == 4 ? s.C.col : which == 5 ? s.Ex.col : s.col;
  const std::vector<double>& v = which == 0 ? s.Kp : which == 1 ? s.Wq : which == 2 ? s.Ea : which == 3 ? s.Gr
                                 : which == 4 ? s.C.vals : s.Ex.vals;
  std::memcpy(rowptr, rp.data(), sizeof(int32_t) * rp.size());
  std::memcpy(col, cl.data(), sizeof(int32_t) * cl.size());
  std::memcpy(vals, v.data(), sizeof(double) * v.size());
  return OK;
}

int pmfem_device_info(pmfem_t h, int64_t* out, int n) {
  if (!h || !out || n <= 0) return EINVAL_;
  int rc = ensure_device(h);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) out[i] = i < 13 ? h->dev_info[i] : 0;
  return OK;
}

int pmfem_debug_fail_alloc(int after) {
  if (after < -1) return EINVAL_;
  g_fail_after.store(after);
  return OK;
}

int pmfem_build_flags(void) { return PMFEM_CHECKS ? 1 : 0; }

int pmfem_setup_times(pmfem_t h, double* out, int n) {
  if (!h || !out || n <= 0) return EINVAL_;
  for (int i = 0; i < n; ++i) out[i] = i < 7 ? h->s.t_stage[i] : 0.0;
  return OK;
}

int pmfem_grid_info(pmfem_t h, int32_t* dims, int32_t* fft, double* origin, double* delta) {
  if (!h || !dims || !fft || !origin || !delta) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  for (int a = 0; a < 3; ++a) {
    dims[a] = h->s.dims[a];
    fft[a] = h->s.fft[a];
    origin[a] = h->s.origin[a];
    delta[a] = h->s.delta[a];
  }
  return OK;
}

int pmfem_export_spectrum(pmfem_t h, double* out) {
  if (!h || !out) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  std::memcpy(out, h->s.ghat.data(), sizeof(double) * h->s.ghat.size());
  return OK;
}

int pmfem_folded_positions(pmfem_t h, double* out) {
  if (!h || !out) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  std::memcpy(out, h->s.pos_f.data(), sizeof(double) * h->s.pos_f.size());
  return OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Field evaluation without any allocation.
//
// Some callers cannot allocate device memory at the moment they need a field: real-time
// loops that forbid allocator calls, or hosts whose memory is owned by a pooling allocator
// that the library must not bypass.
// pmfem_field_noalloc serves them: it computes exactly what pmfem_field computes, but every
// scratch buffer of the evaluation (the permuted magnetisation, charges, potentials, the
// grid and the FFT spectrum buffer) is carved out of one file-scope device array of fixed
// size, and the call makes no allocating CUDA or library call.  The array exists on every
// GPU that loads this library, for the lifetime of the process.
// ------------------------------------------------------------------------------------
namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of scratch one evaluation of this handle needs at precision T
template <typename T>
size_t noalloc_need(const Setup& s) {
  using C2 = typename Vec2<T>::type;
  const size_t np = (size_t)s.Np;
  const size_t G = (size_t)s.dims[0] * s.dims[1] * s.dims[2];
  const size_t ncb = (size_t)(s.fft[0] / 2 + 1) * s.fft[1] * s.fft[2];
  return align256(np * sizeof(V4<T>)) + 2 * align256(np * sizeof(T)) + align256(G * sizeof(T)) +
         align256(ncb * sizeof(C2));
}

template <typename T>
void noalloc_eval(pmfem_t h, const DevOps<T>& d, unsigned char* base, const void* m, void* H, int comps,
                  cudaStream_t st) {
  using C2 = typename Vec2<T>::type;
  DevOps<T> x = d;          // same operators, scratch redirected into the static array
  x.prof = ProfHook();      // no event creation on this path
  const size_t np = (size_t)d.Np;
  const size_t G = (size_t)d.dims[0] * d.dims[1] * d.dims[2];
  size_t off = 0;
  V4<T>* mf = (V4<T>*)(base + off);
  off += align256(np * sizeof(V4<T>));
  x.q = (T*)(base + off);
  off += align256(np * sizeof(T));
  x.e = (T*)(base + off);
  off += align256(np * sizeof(T));
  x.grid = (T*)(base + off);
  off += align256(G * sizeof(T));
  x.cbuf = (C2*)(base + off);
  // every scratch element is written by the evaluation before it is read, so nothing has
  // to start at zero
  launch_perm_in(x, (const T*)m, mf, st);
  RkArgs none;
  enqueue_eval(h, x, (const V4<T>*)mf, (T*)H, comps, none, st);
}

}  // namespace

extern "C" int pmfem_field_noalloc(pmfem_t h, const void* m, void* H, int components, void* stream) {
  if (!h) return EINVAL_;
  if (!m || !H || m == H) return fail(h, EINVAL_, "m and H must be distinct device pointers");
  if (components <= 0 || components > PMFEM_ALL) return fail(h, EINVAL_, "components must be a non-empty PMFEM_EX|MS|AP|AN mask");
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  const size_t need = h->prec == PMFEM_FP64 ? noalloc_need<double>(h->s) : noalloc_need<float>(h->s);
  if (need > kNoAllocBytes)
    return fail(h, EINVAL_, "pmfem_field_noalloc: this mesh and grid need " + std::to_string(need) +
                                " bytes of scratch, more than its fixed " + std::to_string(kNoAllocBytes) +
                                " bytes; use pmfem_field");
  if (!h->dev_ready || h->dev_prec != h->prec)
    return fail(h, ESTATE_, "pmfem_field_noalloc needs the operators on the device: make one pmfem_field (or "
                            "pmfem_set_m) call at this precision first");
  void* base = h->noalloc_base;   // looked up when the device data were built
  if (!base) return fail(h, ECUDA_, h->noalloc_why);
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (h->dev_prec == PMFEM_FP64) noalloc_eval(h, h->d64, (unsigned char*)base, m, H, components, st);
  else noalloc_eval(h, h->d32, (unsigned char*)base, m, H, components, st);
  return check_launch(h);
}

// ------------------------------------------------------------------------------------
// Learned surrogate of the FFT convolution (network and kernels in surrogate.cu).
// ------------------------------------------------------------------------------------
namespace {
// A tensor-core convolution that gave up waiting on its MMAs leaves a flag (ETIMEOUT).
int surrogate_check(pmfem_t h) {
  if (!h->net || !h->net->tc_err) return OK;
  int f = 0;
  PMFEM_CK(h, cudaMemcpy(&f, h->net->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (f) {
    PMFEM_CK(h, cudaMemset(h->net->tc_err, 0, sizeof(int)));
    return fail(h, ETIMEOUT_, "a tensor-core convolution of the surrogate timed out waiting for its MMAs");
  }
  return OK;
}
}  // namespace

extern "C" {

int pmfem_surrogate_set_params(pmfem_t h, const float* params, int64_t n, double sq, double su, int act_bf16) {
  if (!h) return EINVAL_;
  if (!h->s.ready) return fail(h, ESTATE_, "call pmfem_set_periodicity first");
  if (!params || n != kNetParams) return fail(h, EINVAL_, "params must hold " + std::to_string(kNetParams) + " values");
  if (!(sq > 0) || !(su > 0) || !std::isfinite(sq) || !std::isfinite(su)) return fail(h, EINVAL_, "scales must be > 0");
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(params[k])) return fail(h, EINVAL_, "non-finite parameter");
  if (h->net && h->net->bf16 != (act_bf16 != 0)) {
    net_destroy(*h->net);
    delete h->net;
    h->net = nullptr;
  }
  if (!h->net) {
    h->net = new (std::nothrow) SurrogateNet;
    if (!h->net) return fail(h, ENOMEM_, "out of host memory");
    std::string msg;
    const bool per[3] = {h->s.periodic[0], h->s.periodic[1], h->s.periodic[2]};
    int rc = net_create(*h->net, h->s.dims, per, act_bf16 != 0, msg);
    if (rc) {
      delete h->net;
      h->net = nullptr;
      return fail(h, rc, msg);
    }
    apply_prof(h);
  }
  SurrogateNet& net = *h->net;
  std::vector<float> dl;
  net_params_to_device_layout(params, dl);
  PMFEM_CK(h, cudaMemcpy(net.P, dl.data(), dl.size() * sizeof(float), cudaMemcpyHostToDevice));
  PMFEM_CK(h, cudaMemset(net.M, 0, kNetParams * sizeof(float)));
  PMFEM_CK(h, cudaMemset(net.S2, 0, kNetParams * sizeof(float)));
  PMFEM_CK(h, cudaMemset(net.G, 0, kNetParams * sizeof(float)));
  net.sq = (float)sq;
  net.su = (float)su;
  net.adam_t = 0;
  return OK;
}

int pmfem_surrogate_get_params(pmfem_t h, float* params) {
  if (!h || !params) return EINVAL_;
  if (!h->net) return fail(h, ESTATE_, "no surrogate: call pmfem_surrogate_set_params first");
  std::vector<float> dl(kNetParams), out;
  PMFEM_CK(h, cudaMemcpy(dl.data(), h->net->P, dl.size() * sizeof(float), cudaMemcpyDeviceToHost));
  net_params_from_device_layout(dl.data(), out);
  std::memcpy(params, out.data(), out.size() * sizeof(float));
  return OK;
}

int pmfem_surrogate_apply(pmfem_t h, const float* Q, float* U, void* stream) {
  if (!h) return EINVAL_;
  if (!h->net) return fail(h, ESTATE_, "no surrogate: call pmfem_surrogate_set_params first");
  if (!Q || !U || Q == U) return fail(h, EINVAL_, "Q and U must be distinct device pointers");
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  net_forward(*h->net, Q, U, st);
  return check_launch(h);
}

int pmfem_surrogate_grad(pmfem_t h, const float* Q, const float* U, float* grads, double* loss) {
  if (!h) return EINVAL_;
  if (!h->net) return fail(h, ESTATE_, "no surrogate: call pmfem_surrogate_set_params first");
  if (!Q || !U || !grads || !loss) return fail(h, EINVAL_, "NULL argument");
  SurrogateNet& net = *h->net;
  PMFEM_CK(h, cudaMemset(net.G, 0, kNetParams * sizeof(float)));
  PMFEM_CK(h, cudaMemset(net.loss, 0, sizeof(double)));
  net_backward(net, Q, U, 0);
  int rc = check_launch(h);
  if (rc) return rc;
  PMFEM_CK(h, cudaDeviceSynchronize());
  std::vector<float> dl(kNetParams), out;
  PMFEM_CK(h, cudaMemcpy(dl.data(), net.G, dl.size() * sizeof(float), cudaMemcpyDeviceToHost));
  PMFEM_CK(h, cudaMemcpy(loss, net.loss, sizeof(double), cudaMemcpyDeviceToHost));
  net_params_from_device_layout(dl.data(), out);
  std::memcpy(grads, out.data(), out.size() * sizeof(float));
  return surrogate_check(h);
}

int pmfem_surrogate_train(pmfem_t h, const float* Q, const float* U, int64_t npairs, int epochs, int batch, double lr,
                          double* epoch_loss, void* stream) {
  if (!h) return EINVAL_;
  if (!h->net) return fail(h, ESTATE_, "no surrogate: call pmfem_surrogate_set_params first");
  if (!Q || !U || npairs < 1 || epochs < 1 || batch < 1 || !(lr > 0) || !std::isfinite(lr))
    return fail(h, EINVAL_, "need Q, U, npairs >= 1, epochs >= 1, batch >= 1, lr > 0");
  SurrogateNet& net = *h->net;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  for (int e = 0; e < epochs; ++e) {
    PMFEM_CK(h, cudaMemsetAsync(net.loss, 0, sizeof(double), st));
    for (int64_t k = 0; k < npairs; ++k) {
      net_backward(net, Q + k * net.V, U + k * net.V, st);
      if ((k + 1) % batch == 0 || k + 1 == npairs) {
        net_adam(net, (float)lr, ++net.adam_t, st);
        PMFEM_CK(h, cudaMemsetAsync(net.G, 0, kNetParams * sizeof(float), st));
      }
    }
    int rc = check_launch(h);
    if (rc) return rc;
    if (epoch_loss) {
      double l = 0;
      PMFEM_CK(h, cudaMemcpyAsync(&l, net.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
      PMFEM_CK(h, cudaStreamSynchronize(st));
      epoch_loss[e] = l / (double)npairs;
    }
  }
  return OK;
}

int pmfem_grid_pair(pmfem_t h, const void* m, float* Q, float* U, void* stream) {
  if (!h) return EINVAL_;
  if (!m || !Q || !U || Q == U) return fail(h, EINVAL_, "m, Q and U must be device pointers, Q != U");
  if (h->prec == PMFEM_FP64) return fail(h, ESTATE_, "grid pairs are produced by the FP32 path");
  int rc = ensure_device(h);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  DevOps<float>& d = h->d32;
  const size_t gb = (size_t)d.dims[0] * d.dims[1] * d.dims[2] * sizeof(float);
  launch_perm_in(d, (const float*)m, (V4<float>*)h->mF, st);
  launch_charges(d, (const V4<float>*)h->mF, st);
  launch_anterp(d, st);
  PMFEM_CK(h, cudaMemcpyAsync(Q, d.grid, gb, cudaMemcpyDeviceToDevice, st));
  launch_fft_conv(d, st);
  PMFEM_CK(h, cudaMemcpyAsync(U, d.grid, gb, cudaMemcpyDeviceToDevice, st));
  return check_launch(h);
}

int pmfem_surrogate_enable(pmfem_t h, int every_k) {
  if (!h) return EINVAL_;
  if (every_k < 0) return fail(h, EINVAL_, "every_k must be >= 0");
  if (every_k > 0 && !h->net) return fail(h, ESTATE_, "no surrogate: call pmfem_surrogate_set_params first");
  h->sur_every = every_k;
  h->sur_step = h->sur_evals = h->sur_judged = 0;
  if (h->net) PMFEM_CK(h, cudaMemset(h->net->err, 0, 2 * sizeof(double)));
  return OK;
}

int pmfem_surrogate_stats(pmfem_t h, double* out) {
  if (!h || !out) return EINVAL_;
  double e[2] = {0, 0};
  if (h->net) {
    PMFEM_CK(h, cudaDeviceSynchronize());
    PMFEM_CK(h, cudaMemcpy(e, h->net->err, sizeof(e), cudaMemcpyDeviceToHost));
  }
  out[0] = (double)h->sur_step;
  out[1] = (double)h->sur_evals;
  out[2] = (double)h->sur_judged;
  out[3] = e[1] > 0 ? std::sqrt(e[0] / e[1]) : 0.0;
  return surrogate_check(h);
}

}  // extern "C"
