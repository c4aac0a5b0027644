// Batched field evaluation and LLG time stepping of many independent meshes (cells), for
// example the unit cells of a hysteresis sweep, each with its own applied field.
//
// All cells share one device layout: their unknowns are concatenated, each cell starting
// at a multiple of 32 so that every 32-row chunk of a SELL-32 operator belongs to one cell,
// and a chunk -> cell table gives each row its cell's offsets and sizes.  Each pass of the
// field (charges, projection, interpolation + precorrection, gradient + exchange + RK4
// stage) is then ONE launch over the rows of all cells, with the same row code as a single
// mesh (sell.cuh).  The FFT convolution runs once per group of cells with the same grid
// and FFT shape, one block row per cell.  A whole RK4 step (four field evaluations) is
// captured in a CUDA graph and replayed, so a step costs one graph launch on the host.
//
// The batch computes in FP32.  Each cell's operators come from its own set-up, in the
// box order chosen for it (pmfem_set_layout, or pmfem_batch_autotune).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pmfem.h"
#include "device.hpp"
#include "internal.hpp"
#include "sell.cuh"
#include "state.hpp"

using namespace pmfem;

namespace pmfem {
namespace batch_detail {

// Per-cell facts read by the batched kernels (one table entry per cell, device memory).
struct CellDev {
  int64_t node_off;   // first row of the cell in the padded node space (multiple of 32)
  int64_t user_off;   // first unknown of the cell in the caller's concatenated order
  int64_t grid_off;   // first point of the cell's grid in the concatenated grids (multiple of 32)
  int64_t prow_off;   // first row of the cell's projection (its grid points with entries)
  int32_t Np;         // unknowns of the cell
  int32_t G;          // grid points of the cell
  int32_t nprow;      // rows of the cell's projection
  int32_t dims[3];
  int32_t periodic[3];
  float hap[3];       // applied field, A/m
  float gam, alpha;   // gyromagnetic factor gamma0 / (1 + alpha^2) and damping
};

struct FftGroup {
  int dims[3], fft[3];
  std::vector<int> cells;
  const int64_t* boff = nullptr;                  // device: per cell (grid, cbuf, ghat) offsets
  const float2* tw[3] = {nullptr, nullptr, nullptr};
};

// Concatenated SELL-32 operator in host memory (values already in FP32).
struct HostSell {
  int comps = 1;
  std::vector<int32_t> map, len, base;
  std::vector<int64_t> off{0};
  std::vector<int32_t> delta;
  std::vector<std::vector<float>> val;
  bool col16 = true;
  int64_t rows = 0;
  int vw = 1;   // vector width of the cells' layout (the same for every cell)
};

// Append the rows of one cell's operator, starting at row row0 (a multiple of 32, after
// the rows already present); map entries are shifted by map0.
void append_sell(HostSell& G, const SellMatrix& M, int64_t row0, int64_t map0) {
  if (G.val.empty()) G.val.resize(M.comps), G.comps = M.comps, G.vw = M.vw;
  const int64_t pad_rows = row0 - G.rows;   // empty rows padding the previous cell
  for (int64_t r = 0; r < pad_rows; ++r) {
    G.map.push_back(-1);
    G.len.push_back(0);
    G.base.push_back(0);
  }
  for (int64_t c = 0; c < pad_rows / 32; ++c) G.off.push_back(G.off.back());
  const int64_t P0 = G.off.back();
  const int64_t nch = (M.rows + 31) / 32;
  for (int64_t t = 0; t < M.rows; ++t) {
    G.map.push_back((int32_t)(map0 + M.map[t]));
    G.len.push_back(M.len[t]);
    G.base.push_back(M.base[t]);
  }
  for (int64_t t = M.rows; t < 32 * nch; ++t) {   // lanes of the last chunk beyond the cell
    G.map.push_back(-1);
    G.len.push_back(0);
    G.base.push_back(0);
  }
  for (int64_t c = 0; c < nch; ++c) G.off.push_back(P0 + M.off[c + 1]);
  const int64_t P = M.padded();
  if (M.col16)
    G.delta.insert(G.delta.end(), M.d16.begin(), M.d16.end());
  else
    G.delta.insert(G.delta.end(), M.d32.begin(), M.d32.end());
  G.col16 = G.col16 && M.col16;
  for (int k = 0; k < M.comps; ++k)
    for (int64_t o = 0; o < P; ++o) G.val[k].push_back((float)M.val[(size_t)k * P + o]);
  G.rows = row0 + 32 * nch;
}

// process-wide autotuner cache: (grid dims, FFT dims, N' bucket) -> (tile rows, tile planes)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<int, int>> g_tune_cache;

}  // namespace batch_detail
}  // namespace pmfem
using namespace pmfem::batch_detail;

struct pmfem_batch_state {
  std::vector<pmfem_t> cells;
  Error err;
  int p = 3;
  int64_t rows = 0;        // padded node space
  int64_t grows = 0;       // padded grid-point space
  int64_t prows = 0;       // padded row space of the projection (grid points with entries)
  int64_t users = 0;       // sum of N'
  std::vector<int64_t> user_off;
  // device
  bool dev_ready = false;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  std::vector<CellDev> table;
  CellDev* dtable = nullptr;
  const int32_t* node_cell = nullptr;   // per 32-row chunk of the node space
  const int32_t* grid_cell = nullptr;   // per 32-row chunk of the projection's row space
  const int32_t* uidx = nullptr;        // node row -> caller's unknown (global)
  DevSell<float> adj, cor, pro;
  const int32_t* sbase = nullptr;       // stencil base, 3 per node row
  const float* frac = nullptr;
  const int32_t* rowptrX = nullptr;
  const int32_t* colX = nullptr;
  const float* valX = nullptr;
  int64_t nx_exc = 0;
  const int32_t* xnode = nullptr;
  const int64_t* xgrid = nullptr;
  const float* xw = nullptr;
  float* grid = nullptr;
  float2* cbuf = nullptr;
  const float* ghat = nullptr;
  std::vector<FftGroup> groups;
  float *q = nullptr, *e = nullptr;
  V4<float>* m = nullptr;     // state (node rows)
  V4<float>* mA = nullptr;
  V4<float>* mB = nullptr;
  V4<float>* acc = nullptr;
  V4<float>* mF = nullptr;    // permuted input of pmfem_batch_field
  int* flag = nullptr;
  unsigned grid_cap = 0;   // largest grid of a batched launch
  // captured RK4 step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  // per-launch timing (pmfem_batch_profile): an event pair around every kernel launch
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  cudaEvent_t open_ev[pmfem::KID_COUNT] = {};
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  int64_t prof_count[pmfem::KID_COUNT] = {};
  double prof_ms[pmfem::KID_COUNT] = {};
  pmfem::ProfHook prof;
};

namespace pmfem {
namespace {

// ---------------------------------------------------------------- batched kernels
// Row t of the padded node (or grid-point) space belongs to cell cell_of[t / 32]; rows past
// the cell's own count are padding and do nothing.  The kernels walk the row chunks of all
// cells (the work list) in a grid-stride loop over whatever grid they are given.

__global__ void __launch_bounds__(kBlock) kb_perm_in(int64_t rows, const int32_t* __restrict__ node_cell,
                                                    const CellDev* __restrict__ cells,
                                                    const int32_t* __restrict__ uidx, const float* __restrict__ mu,
                                                    V4<float>* __restrict__ m, int* flag) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const CellDev& c = cells[node_cell[t >> 5]];
    if (t - c.node_off >= c.Np) {
      m[t] = V4<float>{0.f, 0.f, 0.f, 0.f};
      continue;
    }
    const int64_t u = uidx[t];
    const V4<float> v{mu[3 * u], mu[3 * u + 1], mu[3 * u + 2], 0.f};
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) atomicOr(flag, FLAG_NONFINITE_IN);
    m[t] = v;
  }
}

__global__ void __launch_bounds__(kBlock) kb_perm_out(int64_t rows, const int32_t* __restrict__ node_cell,
                                                     const CellDev* __restrict__ cells,
                                                     const int32_t* __restrict__ uidx,
                                                     const V4<float>* __restrict__ m, float* __restrict__ mu) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const CellDev& c = cells[node_cell[t >> 5]];
    if (t - c.node_off >= c.Np) continue;
    const int64_t u = uidx[t];
    const V4<float> v = m[t];
    mu[3 * u] = v.x;
    mu[3 * u + 1] = v.y;
    mu[3 * u + 2] = v.z;
  }
}

template <typename CT>
__global__ void __launch_bounds__(kBlock) kb_charges(int64_t rows, const int32_t* __restrict__ node_cell,
                                                    const CellDev* __restrict__ cells, const int32_t* __restrict__ len,
                                                    const int32_t* __restrict__ base, const int64_t* __restrict__ off,
                                                    const CT* __restrict__ dcol, const float* __restrict__ wx,
                                                    const float* __restrict__ wy, const float* __restrict__ wz,
                                                    const float* __restrict__ ex, const float* __restrict__ ey,
                                                    const float* __restrict__ ez, const V4<float>* __restrict__ m,
                                                    float* __restrict__ q, float* __restrict__ e) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const CellDev& c = cells[node_cell[t >> 5]];
    if (t - c.node_off >= c.Np) continue;
    charges_row<float, CT, float>(t, c.node_off, c.Np, len, base, off, dcol, wx, wy, wz, ex, ey, ez, m, q, e);
  }
}

template <typename CT>
__global__ void __launch_bounds__(kBlock) kb_project(int64_t prows, const int32_t* __restrict__ grid_cell,
                                                    const CellDev* __restrict__ cells, const int32_t* __restrict__ map,
                                                    const int32_t* __restrict__ len, const int32_t* __restrict__ base,
                                                    const int64_t* __restrict__ off, const CT* __restrict__ dcol,
                                                    const float* __restrict__ pw, const float* __restrict__ q,
                                                    float* __restrict__ grid) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < prows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const CellDev& c = cells[grid_cell[t >> 5]];
    if (t - c.prow_off >= c.nprow) continue;
    project_row<float, CT, float>(t, map[t], c.node_off, c.Np, len, base, off, dcol, pw, q, grid);
  }
}

__global__ void __launch_bounds__(kBlock) kb_project_exc(int64_t n, const int32_t* __restrict__ node,
                                                        const int64_t* __restrict__ gidx, const float* __restrict__ w,
                                                        const float* __restrict__ q, float* __restrict__ grid) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    atomicAdd(grid + gidx[t], w[t] * q[node[t]]);
  }
}

template <int P, typename CT>
__global__ void __launch_bounds__(kBlock) kb_interp(
    int64_t rows, const int32_t* __restrict__ node_cell, const CellDev* __restrict__ cells,
    const int32_t* __restrict__ map, const int32_t* __restrict__ sbase, const float* __restrict__ frac,
    const float* __restrict__ grid, const int32_t* __restrict__ clen, const int32_t* __restrict__ cbase,
    const int64_t* __restrict__ coff, const CT* __restrict__ dcol, const float* __restrict__ cval,
    const int32_t* __restrict__ rowptrX, const int32_t* __restrict__ colX, const float* __restrict__ valX,
    const float* __restrict__ q, const float* __restrict__ e, const V4<float>* m, float* uw) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const CellDev& c = cells[node_cell[t >> 5]];
    if (t - c.node_off >= c.Np) continue;
    interp_row<float, P, CT, float>(t, map[t], c.node_off, c.Np, sbase, frac, grid + c.grid_off, c.dims[0],
                                    c.dims[1], c.dims[2], c.periodic[0] != 0, c.periodic[1] != 0, c.periodic[2] != 0,
                                    clen, cbase, coff, dcol, cval, rowptrX, colX, valX, q, e, m, uw);
  }
}

template <int MODE, typename CT>
__global__ void __launch_bounds__(kBlock) kb_field(int64_t rows, const int32_t* __restrict__ node_cell,
                                                  const CellDev* __restrict__ cells, const int32_t* __restrict__ len,
                                                  const int32_t* __restrict__ base, const int64_t* __restrict__ off,
                                                  const CT* __restrict__ dcol, const float* __restrict__ gx,
                                                  const float* __restrict__ gy, const float* __restrict__ gz,
                                                  const float* __restrict__ kp,
                                                  const V4<float>* __restrict__ m, const int32_t* __restrict__ uidx,
                                                  float* __restrict__ H, int use_ms, int use_ex, int use_ap,
                                                  V4<float>* __restrict__ m0, V4<float>* __restrict__ mnext,
                                                  V4<float>* __restrict__ accb, float cdt, float bw, int acc_init,
                                                  float dt6, int* flag) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const CellDev& c = cells[node_cell[t >> 5]];
    if (t - c.node_off >= c.Np) continue;
    const float hx = use_ap ? c.hap[0] : 0.f, hy = use_ap ? c.hap[1] : 0.f, hz = use_ap ? c.hap[2] : 0.f;
    field_row<float, MODE, CT, float, float>(t, c.node_off, c.Np, len, base, off, dcol, gx, gy, gz, kp, m,
                                             MODE == 0 ? (int64_t)uidx[t] : 0, H, use_ms, use_ex, hx, hy, hz, m0,
                                             mnext, accb, cdt, bw, acc_init, dt6, c.gam, c.alpha, flag);
  }
}

inline unsigned nblocks(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }
inline unsigned pblocks(const pmfem_batch_state* b, int64_t n) { return std::max(1u, std::min(nblocks(n), b->grid_cap)); }
// (the grid covers every row: measured, a grid capped at a few blocks per SM that strides
// over the rows ran slower on the 64-cell batch, 7.3 -> 8.7 ms per RK4 step)

}  // namespace
}  // namespace pmfem

namespace {

const double kGammaE = 1.76085963023e11;   // electron gyromagnetic ratio, rad/(s T)

void batch_prof_hook(void* ctx, int id, int phase, cudaStream_t st) {
  pmfem_batch_t b = (pmfem_batch_t)ctx;
  if (b->ev_next >= b->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    b->ev_pool.push_back(e);
  }
  cudaEvent_t e = b->ev_pool[b->ev_next++];
  cudaEventRecord(e, st);
  if (phase == 0)
    b->open_ev[id] = e;
  else
    b->recs.push_back({id, b->open_ev[id], e});
}

int bfail(pmfem_batch_t b, int code, const std::string& msg) {
  b->err = {code, msg};
  return code;
}

#define PMFEM_BCK(b, x)                                                                                 \
  do {                                                                                                  \
    cudaError_t e_ = (x);                                                                               \
    if (e_ != cudaSuccess) return bfail(b, ECUDA_, std::string(#x) + ": " + cudaGetErrorString(e_));   \
  } while (0)

int balloc(pmfem_batch_t b, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return bfail(b, e == cudaErrorMemoryAllocation ? ENOMEM_ : ECUDA_,
                 std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  b->allocs.push_back(*p);
  return OK;
}

template <typename X>
int bupload(pmfem_batch_t b, const X* src, size_t n, const X** out) {
  void* p;
  int rc = balloc(b, &p, n * sizeof(X));
  if (rc) return rc;
  if (n) PMFEM_BCK(b, cudaMemcpy(p, src, n * sizeof(X), cudaMemcpyHostToDevice));
  *out = (const X*)p;
  return OK;
}

void free_batch_device(pmfem_batch_t b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  b->adj = b->cor = b->pro = DevSell<float>();
  b->groups.clear();
  b->dtable = nullptr;
  b->dev_ready = false;
}

int upload_hsell(pmfem_batch_t b, HostSell& H, DevSell<float>& D) {
  int rc;
  D.rows = H.rows;
  D.col16 = H.col16;
  if ((rc = bupload(b, H.map.data(), H.map.size(), &D.map))) return rc;
  if ((rc = bupload(b, H.len.data(), H.len.size(), &D.len))) return rc;
  if ((rc = bupload(b, H.base.data(), H.base.size(), &D.base))) return rc;
  for (int64_t o : H.off)
    if (o % H.vw) return bfail(b, ESTATE_, "internal: SELL chunk offset not a multiple of the vector width");
  if ((rc = bupload(b, H.off.data(), H.off.size(), &D.off))) return rc;
  if (H.col16) {
    std::vector<int16_t> d16(H.delta.begin(), H.delta.end());
    const int16_t* p;
    if ((rc = bupload(b, d16.data(), d16.size(), &p))) return rc;
    D.delta = p;
  } else {
    const int32_t* p;
    if ((rc = bupload(b, H.delta.data(), H.delta.size(), &p))) return rc;
    D.delta = p;
  }
  for (int k = 0; k < H.comps; ++k)
    if ((rc = bupload(b, H.val[k].data(), H.val[k].size(), &D.val[k]))) return rc;
  return OK;
}

// Concatenate the cells' layouts (each built from its own set-up) and upload them.
int build_batch_device(pmfem_batch_t b) {
  const int n = (int)b->cells.size();
  b->table.assign(n, CellDev{});
  HostSell adj, cor, pro;
  std::vector<int32_t> uidx, sbase, node_cell, grid_cell, rowptrX{0}, colX, xnode;
  std::vector<float> frac, valX, xw, ghat;
  std::vector<int64_t> xgrid;
  std::map<std::vector<int>, int> gkey;
  std::vector<std::vector<int64_t>> goffs;
  int64_t row = 0, grow = 0, prow = 0, user = 0, cb = 0, gh = 0;
  b->user_off.assign(n + 1, 0);
  for (int c = 0; c < n; ++c) {
    const Setup& s = b->cells[c]->s;
    Layout L;
    Error err;
    int rc = build_layout(s, L, err);
    if (rc) return bfail(b, rc, "cell " + std::to_string(c) + ": " + err.msg);
    CellDev& d = b->table[c];
    const int64_t Np = s.Np, G = (int64_t)s.dims[0] * s.dims[1] * s.dims[2];
    const int64_t nch = (Np + 31) / 32, gch = (G + 31) / 32;
    d.node_off = row;
    d.user_off = user;
    d.grid_off = grow;
    d.Np = (int32_t)Np;
    d.G = (int32_t)G;
    d.prow_off = prow;
    d.nprow = (int32_t)L.pro.rows;
    for (int a = 0; a < 3; ++a) {
      d.dims[a] = s.dims[a];
      d.periodic[a] = s.periodic[a] ? 1 : 0;
      d.hap[a] = (float)b->cells[c]->hap[a];
    }
    d.gam = (float)(kMu0 * kGammaE / (1.0 + s.alpha * s.alpha));
    d.alpha = (float)s.alpha;
    append_sell(adj, L.adj, row, row);
    append_sell(cor, L.cor, row, row);
    append_sell(pro, L.pro, prow, grow);   // rows: the grid points with entries; map: grid points
    for (int64_t i = 0; i < 32 * nch; ++i) {
      const bool in = i < Np;
      uidx.push_back(in ? (int32_t)(user + L.perm[i]) : 0);
      for (int a = 0; a < 3; ++a) {
        sbase.push_back(in ? L.base[3 * i + a] : 0);
        frac.push_back(in ? (float)L.frac[3 * i + a] : 0.f);
      }
      const int64_t x0 = in ? L.Ex.rowptr[i] : 0, x1 = in ? L.Ex.rowptr[i + 1] : 0;
      for (int64_t q = x0; q < x1; ++q) {
        colX.push_back((int32_t)(row + L.Ex.col[q]));
        for (int a = 0; a < 3; ++a) valX.push_back((float)L.Ex.vals[3 * q + a]);
      }
      rowptrX.push_back((int32_t)colX.size());
    }
    for (size_t k = 0; k < L.xnode.size(); ++k) {
      xnode.push_back((int32_t)(row + L.xnode[k]));
      xgrid.push_back(grow + L.xgrid[k]);
      xw.push_back((float)L.xw[k]);
    }
    for (int64_t k = 0; k < nch; ++k) node_cell.push_back(c);
    const int64_t pch = (L.pro.rows + 31) / 32;
    for (int64_t k = 0; k < pch; ++k) grid_cell.push_back(c);
    const double scale = 1.0 / ((double)s.fft[0] * s.fft[1] * s.fft[2]);
    for (double g : s.ghat) ghat.push_back((float)(g * scale));
    const std::vector<int> key{s.dims[0], s.dims[1], s.dims[2], s.fft[0], s.fft[1], s.fft[2]};
    auto it = gkey.find(key);
    if (it == gkey.end()) {
      it = gkey.emplace(key, (int)b->groups.size()).first;
      FftGroup g;
      for (int a = 0; a < 3; ++a) g.dims[a] = s.dims[a], g.fft[a] = s.fft[a];
      b->groups.push_back(g);
      goffs.emplace_back();
    }
    b->groups[it->second].cells.push_back(c);
    goffs[it->second].insert(goffs[it->second].end(), {grow, cb, gh});
    cb += (int64_t)(s.fft[0] / 2 + 1) * s.fft[1] * s.fft[2];
    gh += (int64_t)s.ghat.size();
    row += 32 * nch;
    grow += 32 * gch;
    prow += 32 * pch;
    user += Np;
    b->user_off[c + 1] = user;
  }
  b->rows = row;
  b->grows = grow;
  b->prows = prow;
  b->users = user;
  int rc;
  if ((rc = upload_hsell(b, adj, b->adj))) return rc;
  adj = HostSell();
  if ((rc = upload_hsell(b, cor, b->cor))) return rc;
  cor = HostSell();
  if ((rc = upload_hsell(b, pro, b->pro))) return rc;
  pro = HostSell();
  const CellDev* tp;
  if ((rc = bupload(b, b->table.data(), b->table.size(), &tp))) return rc;
  b->dtable = const_cast<CellDev*>(tp);
  if ((rc = bupload(b, node_cell.data(), node_cell.size(), &b->node_cell))) return rc;
  if ((rc = bupload(b, grid_cell.data(), grid_cell.size(), &b->grid_cell))) return rc;
  if ((rc = bupload(b, uidx.data(), uidx.size(), &b->uidx))) return rc;
  if ((rc = bupload(b, sbase.data(), sbase.size(), &b->sbase))) return rc;
  if ((rc = bupload(b, frac.data(), frac.size(), &b->frac))) return rc;
  if ((rc = bupload(b, rowptrX.data(), rowptrX.size(), &b->rowptrX))) return rc;
  if ((rc = bupload(b, colX.data(), colX.size(), &b->colX))) return rc;
  if ((rc = bupload(b, valX.data(), valX.size(), &b->valX))) return rc;
  b->nx_exc = (int64_t)xnode.size();
  if ((rc = bupload(b, xnode.data(), xnode.size(), &b->xnode))) return rc;
  if ((rc = bupload(b, xgrid.data(), xgrid.size(), &b->xgrid))) return rc;
  if ((rc = bupload(b, xw.data(), xw.size(), &b->xw))) return rc;
  if ((rc = bupload(b, ghat.data(), ghat.size(), &b->ghat))) return rc;
  for (size_t k = 0; k < b->groups.size(); ++k) {
    FftGroup& g = b->groups[k];
    if ((rc = bupload(b, goffs[k].data(), goffs[k].size(), &g.boff))) return rc;
    for (int a = 0; a < 3; ++a) {
      const int F = g.fft[a];
      std::vector<float2> tw(F);
      for (int j = 0; j < F; ++j) {
        const double ang = 2.0 * kPi * j / F;
        tw[j].x = (float)std::cos(ang);
        tw[j].y = (float)(-std::sin(ang));
      }
      if ((rc = bupload(b, tw.data(), tw.size(), &g.tw[a]))) return rc;
    }
  }
  void* p;
  const size_t sv = (size_t)row * sizeof(V4<float>), ss = (size_t)row * sizeof(float);
  if ((rc = balloc(b, &p, ss))) return rc;
  b->q = (float*)p;
  if ((rc = balloc(b, &p, ss))) return rc;
  b->e = (float*)p;
  if ((rc = balloc(b, &p, (size_t)grow * sizeof(float)))) return rc;
  b->grid = (float*)p;
  if ((rc = balloc(b, &p, (size_t)cb * sizeof(float2)))) return rc;
  b->cbuf = (float2*)p;
  V4<float>** vs[5] = {&b->m, &b->mA, &b->mB, &b->acc, &b->mF};
  for (V4<float>** v : vs) {
    if ((rc = balloc(b, &p, sv))) return rc;
    *v = (V4<float>*)p;
    PMFEM_BCK(b, cudaMemset(p, 0, sv));
  }
  if ((rc = balloc(b, &p, sizeof(int)))) return rc;
  b->flag = (int*)p;
  PMFEM_BCK(b, cudaMemset(b->flag, 0, sizeof(int)));
  PMFEM_BCK(b, cudaMemset(b->q, 0, ss));
  PMFEM_BCK(b, cudaMemset(b->e, 0, ss));
  b->dev_ready = true;
  return OK;
}

int ensure_batch(pmfem_batch_t b) {
  if (b->dev_ready) return OK;
  free_batch_device(b);
  if (!b->stream) PMFEM_BCK(b, cudaStreamCreate(&b->stream));
  int dev = 0, sms = 0;
  PMFEM_BCK(b, cudaGetDevice(&dev));
  PMFEM_BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->grid_cap = 0xFFFFFFFFu;   // one thread per row (see pblocks)
  (void)sms;
  int rc = build_batch_device(b);
  if (rc) free_batch_device(b);
  return rc;
}

}  // namespace

namespace {

template <typename F>
void with_cols(const DevSell<float>& M, F&& f) {
  if (M.col16)
    f((const int16_t*)M.delta);
  else
    f((const int32_t*)M.delta);
}

// One field evaluation of every cell (the single-mesh sequence of enqueue_eval), with the
// RK4 stage epilogue selected by rk.mode.
void batch_eval(pmfem_batch_t b, const V4<float>* m, float* H, int comps, const RkArgs& rk, cudaStream_t st) {
  const unsigned nb = pblocks(b, b->rows);
  const DevSell<float>& A = b->adj;
  if (comps & PMFEM_MS) {
    b->prof.begin(KID_CHARGES, st);
    with_cols(A, [&](auto dcol) {
      using CT = std::remove_cv_t<std::remove_pointer_t<decltype(dcol)>>;
      kb_charges<CT><<<nb, kBlock, 0, st>>>(b->rows, b->node_cell, b->dtable, A.len, A.base, A.off, dcol, A.val[0],
                                            A.val[1], A.val[2], A.val[3], A.val[4], A.val[5], m, b->q, b->e);
    });
    b->prof.end(KID_CHARGES, st);
    b->prof.begin(KID_ANTERP, st);
    const DevSell<float>& Pm = b->pro;
    // a cell's projection may hold only its grid points with entries: then clear the grids first
    if (b->prows < b->grows) cudaMemsetAsync(b->grid, 0, (size_t)b->grows * sizeof(float), st);
    if (b->prows > 0)
      with_cols(Pm, [&](auto dcol) {
        using CT = std::remove_cv_t<std::remove_pointer_t<decltype(dcol)>>;
        kb_project<CT><<<pblocks(b, b->prows), kBlock, 0, st>>>(b->prows, b->grid_cell, b->dtable, Pm.map, Pm.len,
                                                             Pm.base, Pm.off, dcol, Pm.val[0], b->q, b->grid);
      });
    if (b->nx_exc > 0)
      kb_project_exc<<<pblocks(b, b->nx_exc), kBlock, 0, st>>>(b->nx_exc, b->xnode, b->xgrid, b->xw, b->q, b->grid);
    b->prof.end(KID_ANTERP, st);
    for (const FftGroup& g : b->groups) {
      FftArgs<float> a;
      a.grid = b->grid;
      a.cbuf = b->cbuf;
      a.ghat = b->ghat;
      for (int k = 0; k < 3; ++k) {
        a.dims[k] = g.dims[k];
        a.fft[k] = g.fft[k];
        a.tw[k] = g.tw[k];
      }
      a.boff = g.boff;
      a.count = (unsigned)g.cells.size();
      launch_fft(a, b->prof, st);
    }
    b->prof.begin(KID_INTERP, st);
    const DevSell<float>& C = b->cor;
    with_cols(C, [&](auto dcol) {
      using CT = std::remove_cv_t<std::remove_pointer_t<decltype(dcol)>>;
      auto go = [&](auto kernel) {
        kernel<<<nb, kBlock, 0, st>>>(b->rows, b->node_cell, b->dtable, C.map, b->sbase, b->frac, b->grid, C.len,
                                      C.base, C.off, dcol, C.val[0], b->rowptrX, b->colX, b->valX, b->q, b->e, m,
                                      reinterpret_cast<float*>(const_cast<V4<float>*>(m)) + 3);   // u -> lane 3
      };
      switch (b->p) {
        case 2: go(kb_interp<3, CT>); break;
        case 3: go(kb_interp<4, CT>); break;
        case 4: go(kb_interp<5, CT>); break;
        default: go(kb_interp<6, CT>); break;
      }
    });
    b->prof.end(KID_INTERP, st);
  }
  const int use_ms = (comps & PMFEM_MS) ? 1 : 0, use_ex = (comps & PMFEM_EX) ? 1 : 0, use_ap = (comps & PMFEM_AP) ? 1 : 0;
  with_cols(A, [&](auto dcol) {
    using CT = std::remove_cv_t<std::remove_pointer_t<decltype(dcol)>>;
    auto go = [&](auto kernel) {
      kernel<<<nb, kBlock, 0, st>>>(b->rows, b->node_cell, b->dtable, A.len, A.base, A.off, dcol, A.val[6], A.val[7],
                                    A.val[8], A.val[9], m, b->uidx, H, use_ms, use_ex, use_ap,
                                    (V4<float>*)rk.m0, (V4<float>*)rk.mnext, (V4<float>*)rk.acc, (float)rk.cdt,
                                    (float)rk.bw, rk.acc_init, (float)rk.dt6, b->flag);
    };
    b->prof.begin(KID_FIELD, st);
    if (rk.mode == 0)
      go(kb_field<0, CT>);
    else if (rk.mode == 1)
      go(kb_field<1, CT>);
    else
      go(kb_field<2, CT>);
    b->prof.end(KID_FIELD, st);
  });
}

// One classical RK4 step of every cell (the stages of run_llg in api.cu).
void batch_rk_step(pmfem_batch_t b, double dt, cudaStream_t st) {
  RkArgs rk;
  rk.m0 = b->m;
  rk.acc = b->acc;
  rk.mode = 1;
  rk.cdt = 0.5 * dt, rk.bw = 1.0, rk.acc_init = 1, rk.mnext = b->mA;
  batch_eval(b, b->m, nullptr, PMFEM_ALL, rk, st);
  rk.cdt = 0.5 * dt, rk.bw = 2.0, rk.acc_init = 0, rk.mnext = b->mB;
  batch_eval(b, b->mA, nullptr, PMFEM_ALL, rk, st);
  rk.cdt = dt, rk.bw = 2.0, rk.acc_init = 0, rk.mnext = b->mA;
  batch_eval(b, b->mB, nullptr, PMFEM_ALL, rk, st);
  rk.mode = 2;
  rk.dt6 = dt / 6.0;
  batch_eval(b, b->mA, nullptr, PMFEM_ALL, rk, st);
}

int capture_step(pmfem_batch_t b, double dt) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  // FFT kernels opt into large shared memory outside the capture
  for (const FftGroup& g : b->groups) {
    FftArgs<float> a;
    a.grid = b->grid;
    a.cbuf = b->cbuf;
    a.ghat = b->ghat;
    for (int k = 0; k < 3; ++k) a.dims[k] = g.dims[k], a.fft[k] = g.fft[k], a.tw[k] = g.tw[k];
    a.boff = g.boff;
    a.count = (unsigned)g.cells.size();
    launch_fft(a, ProfHook(), b->stream);
  }
  PMFEM_BCK(b, cudaStreamSynchronize(b->stream));
  cudaStream_t cs;
  PMFEM_BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    batch_rk_step(b, dt, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, ECUDA_, std::string("RK4 step capture failed: ") + cudaGetErrorString(e));
  }
  b->graph_dt = dt;
  return OK;
}

}  // namespace

extern "C" {

int pmfem_batch_create(pmfem_batch_t* out, const pmfem_t* cells, int n) {
  if (!out) return EINVAL_;
  *out = nullptr;
  if (!cells || n < 1) return EINVAL_;
  for (int c = 0; c < n; ++c) {
    if (!cells[c]) return EINVAL_;
    if (!cells[c]->s.ready) return ESTATE_;
    if (cells[c]->s.p != cells[0]->s.p) return EINVAL_;
  }
  pmfem_batch_t b = new (std::nothrow) pmfem_batch_state;
  if (!b) return ENOMEM_;
  b->cells.assign(cells, cells + n);
  b->p = cells[0]->s.p;
  b->user_off.assign(n + 1, 0);
  for (int c = 0; c < n; ++c) b->user_off[c + 1] = b->user_off[c] + cells[c]->s.Np;
  b->users = b->user_off[n];
  *out = b;
  return OK;
}

int pmfem_batch_profile(pmfem_batch_t b, int enable) {
  if (!b) return EINVAL_;
  b->prof_on = enable != 0;
  b->recs.clear();
  b->ev_next = 0;
  for (int i = 0; i < KID_COUNT; ++i) b->prof_count[i] = 0, b->prof_ms[i] = 0;
  if (b->prof_on) {
    b->prof.fn = batch_prof_hook;
    b->prof.ctx = b;
  } else {
    b->prof = ProfHook();
  }
  return OK;
}

int pmfem_batch_profile_read(pmfem_batch_t b, int64_t* counts, double* total_ms, int n) {
  if (!b || !counts || !total_ms || n <= 0) return EINVAL_;
  PMFEM_BCK(b, cudaDeviceSynchronize());
  for (auto& r : b->recs) {
    float ms = 0;
    PMFEM_BCK(b, cudaEventElapsedTime(&ms, r.a, r.b));
    b->prof_count[r.id] += 1;
    b->prof_ms[r.id] += ms;
  }
  b->recs.clear();
  b->ev_next = 0;
  for (int i = 0; i < n; ++i) {
    counts[i] = i < KID_COUNT ? b->prof_count[i] : 0;
    total_ms[i] = i < KID_COUNT ? b->prof_ms[i] : 0.0;
  }
  return OK;
}

int pmfem_batch_destroy(pmfem_batch_t b) {
  if (!b) return EINVAL_;
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
  free_batch_device(b);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return OK;
}

const char* pmfem_batch_last_error(pmfem_batch_t b) { return b ? b->err.msg.c_str() : "batch is NULL"; }

int pmfem_batch_offsets(pmfem_batch_t b, int64_t* offsets) {
  if (!b || !offsets) return EINVAL_;
  for (size_t c = 0; c < b->user_off.size(); ++c) offsets[c] = b->user_off[c];
  return OK;
}

int pmfem_batch_tiles(pmfem_batch_t b, int32_t* tiles) {
  if (!b || !tiles) return EINVAL_;
  for (size_t c = 0; c < b->cells.size(); ++c) {
    const Setup& s = b->cells[c]->s;
    int ty = s.tile_y > 0 ? s.tile_y : 8, tz = s.tile_z > 0 ? s.tile_z : 4;
    while (ty > 1 && s.dims[1] % ty) ty /= 2;   // the rule of build_layout
    while (tz > 1 && s.dims[2] % tz) tz /= 2;
    tiles[2 * c] = std::min(ty, s.dims[1]);
    tiles[2 * c + 1] = std::min(tz, s.dims[2]);
  }
  return OK;
}

int pmfem_batch_set_applied_field(pmfem_batch_t b, int c, double Hx, double Hy, double Hz, void* stream) {
  if (!b) return EINVAL_;
  if (c < 0 || c >= (int)b->cells.size()) return bfail(b, EINVAL_, "cell index out of range");
  if (!(std::isfinite(Hx) && std::isfinite(Hy) && std::isfinite(Hz))) return bfail(b, EINVAL_, "field not finite");
  b->cells[c]->hap[0] = Hx, b->cells[c]->hap[1] = Hy, b->cells[c]->hap[2] = Hz;
  if (!b->dev_ready) return OK;   // read at the next build
  CellDev& d = b->table[c];
  d.hap[0] = (float)Hx, d.hap[1] = (float)Hy, d.hap[2] = (float)Hz;
  cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
  PMFEM_BCK(b, cudaMemcpyAsync(&b->dtable[c].hap, d.hap, sizeof(d.hap), cudaMemcpyHostToDevice, st));
  return OK;
}

int pmfem_batch_field(pmfem_batch_t b, const void* m, void* H, int components, void* stream) {
  if (!b) return EINVAL_;
  if (!m || !H || components < 0 || components > PMFEM_ALL) return bfail(b, EINVAL_, "bad m, H or components");
  int rc = ensure_batch(b);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
  kb_perm_in<<<pblocks(b, b->rows), kBlock, 0, st>>>(b->rows, b->node_cell, b->dtable, b->uidx, (const float*)m, b->mF,
                                                  b->flag);
  batch_eval(b, b->mF, (float*)H, components, RkArgs(), st);
  PMFEM_BCK(b, cudaGetLastError());
  return OK;
}

int pmfem_batch_set_m(pmfem_batch_t b, const void* m, void* stream) {
  if (!b) return EINVAL_;
  if (!m) return bfail(b, EINVAL_, "m is NULL");
  int rc = ensure_batch(b);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
  kb_perm_in<<<pblocks(b, b->rows), kBlock, 0, st>>>(b->rows, b->node_cell, b->dtable, b->uidx, (const float*)m, b->m,
                                                  b->flag);
  PMFEM_BCK(b, cudaGetLastError());
  return OK;
}

int pmfem_batch_get_m(pmfem_batch_t b, void* m, void* stream) {
  if (!b) return EINVAL_;
  if (!m) return bfail(b, EINVAL_, "m is NULL");
  int rc = ensure_batch(b);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
  kb_perm_out<<<pblocks(b, b->rows), kBlock, 0, st>>>(b->rows, b->node_cell, b->dtable, b->uidx, b->m, (float*)m);
  PMFEM_BCK(b, cudaGetLastError());
  return OK;
}

int pmfem_batch_llg_step(pmfem_batch_t b, double dt, int nsteps, void* stream) {
  if (!b) return EINVAL_;
  if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return bfail(b, EINVAL_, "need dt > 0 and nsteps >= 0");
  int rc = ensure_batch(b);
  if (rc) return rc;
  cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
  if (nsteps == 0) return OK;
  if (b->prof_on) {   // launch by launch, each timed on the stream
    for (int k = 0; k < nsteps; ++k) batch_rk_step(b, dt, st);
    PMFEM_BCK(b, cudaGetLastError());
    return OK;
  }
  if (!b->graph || b->graph_dt != dt) {
    // the capture reads the state buffers by address only: order it after the caller's work
    PMFEM_BCK(b, cudaStreamSynchronize(st));
    if ((rc = capture_step(b, dt))) return rc;
  }
  for (int k = 0; k < nsteps; ++k) PMFEM_BCK(b, cudaGraphLaunch(b->graph, st));
  return OK;
}

int pmfem_batch_sync(pmfem_batch_t b) {
  if (!b) return EINVAL_;
  if (!b->dev_ready) return OK;
  PMFEM_BCK(b, cudaDeviceSynchronize());
  int flag = 0;
  PMFEM_BCK(b, cudaMemcpy(&flag, b->flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    PMFEM_BCK(b, cudaMemset(b->flag, 0, sizeof(int)));
    return bfail(b, ENONFINITE_, (flag & FLAG_NONFINITE_IN) ? "non-finite magnetisation input"
                                                            : "non-finite field result");
  }
  return OK;
}

int pmfem_batch_autotune(pmfem_batch_t b, int reps) {
  if (!b) return EINVAL_;
  if (reps < 1 || reps > 100) return bfail(b, EINVAL_, "reps must be in [1, 100]");
  static const int cand[][2] = {{8, 4}, {8, 2}, {4, 4}, {16, 2}, {4, 2}};
  free_batch_device(b);   // room for the cells' own device data while they are timed
  for (pmfem_t h : b->cells) {
    Setup& s = h->s;
    const auto key = std::make_tuple(s.dims[0], s.dims[1], s.dims[2], s.fft[0], s.fft[1], s.fft[2],
                                     (int)std::lround(4.0 * std::log2((double)std::max<int64_t>(s.Np, 1))));
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        pmfem_set_layout(h, it->second.first, it->second.second, s.sort_window, s.col_bits);
        continue;
      }
    }
    const int prec = h->prec;
    pmfem_set_precision(h, PMFEM_FP32);
    void *m = nullptr, *H = nullptr;
    const size_t bytes = 3 * (size_t)s.Np * sizeof(float);
    if (cudaMalloc(&m, bytes) != cudaSuccess || cudaMalloc(&H, bytes) != cudaSuccess) {
      cudaFree(m);
      pmfem_set_precision(h, prec);
      return bfail(b, ENOMEM_, "autotune: no device memory for the timing buffers");
    }
    cudaMemset(m, 0, bytes);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bi = 0, rc = OK;
    for (int k = 0; k < 5 && rc == OK; ++k) {
      if ((rc = pmfem_set_layout(h, cand[k][0], cand[k][1], s.sort_window, s.col_bits))) break;
      if ((rc = pmfem_field(h, m, H, PMFEM_ALL, nullptr))) break;   // builds the device data, warms up
      cudaEventRecord(e0, h->stream);
      for (int r = 0; r < reps && rc == OK; ++r) rc = pmfem_field(h, m, H, PMFEM_ALL, nullptr);
      cudaEventRecord(e1, h->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = ECUDA_;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == OK && ms < best) best = ms, bi = k;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(m);
    cudaFree(H);
    if (rc) {
      pmfem_set_precision(h, prec);
      return bfail(b, rc, std::string("autotune: ") + pmfem_last_error(h));
    }
    pmfem_set_layout(h, cand[bi][0], cand[bi][1], s.sort_window, s.col_bits);   // also frees the cell's device data
    pmfem_set_precision(h, prec);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {cand[bi][0], cand[bi][1]};
  }
  return OK;
}

}  // extern "C"
