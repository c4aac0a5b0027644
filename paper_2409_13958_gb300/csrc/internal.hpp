// Internal declarations of libpmfem: host set-up state and helpers.
// Not part of the public ABI (see include/pmfem.h).
#pragma once

#include <array>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "setup_math.hpp"

namespace pmfem {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4e-7 * kPi;

// status codes (mirror of pmfem.h)
enum Status : int { OK = 0, EINVAL_ = -1, ENOMEM_ = -2, ECUDA_ = -3, EMESH_ = -4,
                    ENONFINITE_ = -5, ETIMEOUT_ = -6, ESTATE_ = -7,
                    ENOCONV_ = -8 };

struct Error {
  int code = 0;
  std::string msg;
};

// Compressed sparse rows with `comps` values per entry (row-major per entry).
struct Csr {
  int64_t rows = 0;
  int comps = 1;
  std::vector<int32_t> rowptr;  // rows + 1
  std::vector<int32_t> col;
  std::vector<double> vals;     // nnz * comps
  int64_t nnz() const { return (int64_t)col.size(); }
};

struct Setup {
  // ---- mesh and material
  int64_t N = 0, T = 0;
  std::vector<double> xyz;      // N x 3
  std::vector<int32_t> tets;    // T x 4, positively oriented
  double Ms = 0, A = 0, alpha = 0;
  std::vector<double> A_tet;    // T exchange stiffness per tetrahedron (empty: A everywhere)
  // ---- anisotropy per grain (pmfem_set_anisotropy): grain of every tetrahedron and, per
  // grain, axes a1 a2 a3 (9, rows), c1 = -2 K1/(mu0 Ms), u (3), cu = 2 Ku/(mu0 Ms), 2 pads
  std::vector<int32_t> tet_grain;
  std::vector<double> grain_tab;
  // ---- AIM settings (0 = default)
  int dims_req[3] = {0, 0, 0};
  int p = 3;
  int near_boxes = 3;
  double near_elem_factor = 0.0;
  // ---- set-up on the GPU (pmfem_set_setup_device): PGF spectrum, near-element integrals and
  // point precorrection evaluated by CUDA kernels in FP64 on the current device
  bool setup_gpu = false;
  // ---- device layout tuning (0 = default)
  int tile_y = 0, tile_z = 0, sort_window = 0, col_bits = 0;
  // ---- periodicity
  double L[3] = {0, 0, 0};
  bool periodic[3] = {false, false, false};
  // ---- pairing (Sec. 2.2)
  int64_t Np = 0;
  std::vector<int32_t> lca;     // N: node -> unknown
  std::vector<int32_t> roots;   // Np: unknown -> node
  std::vector<double> pos_f;    // Np x 3 folded positions (Eq. 18)
  double r0[3] = {0, 0, 0};
  // ---- local operators on the adjacency pattern (Eqs. 8-12, 14a, 14d)
  std::vector<int32_t> rowptr, col;  // adjacency of unknowns (shared pattern)
  std::vector<double> V;             // lumped nodal volumes
  std::vector<double> Kp;            // nnz    exchange, scaled
  std::vector<double> Wq;            // nnz*3  charges, scaled by Ms
  std::vector<double> Ea;            // nnz*3  near-element correction, scaled by Ms
  std::vector<double> Gr;            // nnz*3  gradient, scaled by -1/(4 pi V_n)
  Csr C;                             // point precorrection (step 4)
  Csr Ex;                            // near-element entries outside the adjacency pattern
  // ---- boundary and sizes
  std::vector<int32_t> bfaces;       // F x 3 original node indices, outward orientation
  double mean_edge = 0;
  // ---- grid (Eq. 16)
  int dims[3] = {0, 0, 0};
  int fft[3] = {0, 0, 0};
  double origin[3] = {0, 0, 0};
  double delta[3] = {0, 0, 0};
  std::vector<int32_t> base;         // Np x 3 unwrapped stencil start
  std::vector<double> frac;          // Np x 3 local coordinate s = t - base
  std::vector<double> ghat;          // (F0/2+1)(F1/2+1)(F2/2+1), x fastest, unscaled
  std::vector<int32_t> box;          // Np x 3 grid box of each unknown (folded position)
  bool ready = false;
  // ---- wall seconds of the set-up stages (pmfem_setup_times): pairing + fold, local
  // operators, grid, PGF spectrum, near elements, point precorrection, device layout + upload
  double t_stage[7] = {0, 0, 0, 0, 0, 0, 0};
};

// Device-side layout: unknowns re-ordered by grid box (z-major, then y, then x) so that
// sparse rows gather from nearby indices, and every sparse operator stored in SELL-32
// for one-thread-per-row kernels: element j of the row handled by thread t sits at
// off[t / 32] + 32 j + t % 32.  Columns are stored as deltas to a per-row base, 16-bit
// when every delta of the operator fits, else 32-bit.
struct SellMatrix {
  int64_t rows = 0;
  int vw = 1;                        // values per lane and step: element j of a row sits at
                                     // off[c] + ((j / vw) * 32 + lane) * vw + j % vw
  std::vector<int32_t> map;          // thread -> row (identity unless rows were length-sorted)
  std::vector<int32_t> len;          // per thread
  std::vector<int32_t> base;         // per thread: column = base + delta
  std::vector<int64_t> off;          // chunks + 1
  bool col16 = true;
  std::vector<int16_t> d16;
  std::vector<int32_t> d32;
  std::vector<double> val;           // comps x padded size, component-major
  int comps = 1;
  int64_t padded() const { return off.empty() ? 0 : off.back(); }
};

struct Layout {
  int TY = 1, TZ = 1;                // box rows / planes per tile in the box order (1: plain)
  int pl = 1, pr = 2;                // stencil reach below / above a node's box
  std::vector<int32_t> perm;         // internal -> user unknown
  std::vector<int32_t> box;          // Np x 3, internal order
  std::vector<int32_t> bstart;       // (boxes + 1): first internal node of each box
  std::vector<int32_t> rowptr, col;  // adjacency, internal numbering
  std::vector<double> Wq, Ea, Gr, Kp;
  std::vector<int32_t> base;
  std::vector<double> frac;
  std::vector<int64_t> cptr;         // Np + 1: start of each row's precorrection values
  std::vector<double> cval;          // values in (dz, dy, x-segment, node) order
  std::vector<int32_t> ccol;         // their source nodes
  Csr Ex;                            // near-element entries beyond the pattern, internal
  SellMatrix adj;                    // 10 components: W^q (3), E (3), gradient (3), exchange
  SellMatrix cor;                    // point precorrection, rows length-sorted in windows
  SellMatrix pro;                    // projection P^T: rows = grid points
  std::vector<int32_t> xnode;        // projection exceptions: node, grid index, weight
  std::vector<int64_t> xgrid;
  std::vector<double> xw;
  int64_t box_index(int x, int y, int z, const int N[3]) const {
    const int ty = y / TY, yi = y % TY, tz = z / TZ, zi = z % TZ;
    return ((((int64_t)tz * (N[1] / TY) + ty) * TZ + zi) * TY + yi) * N[0] + x;
  }
};
#ifndef PMFEM_COR_VW
#define PMFEM_COR_VW 8   // vector width of the precorrection's SELL layout (also read by the kernels)
#endif
int build_layout(const Setup& s, Layout& L, Error& err);
// Centre of a row's columns and the columns' deltas to it, both modulo n (|delta| <= n/2);
// returns the largest |delta|.
int64_t centre_deltas(const int32_t* cols, int64_t len, int32_t ref, int64_t n, int32_t* base, int32_t* delta);

// set-up stages (host, FP64); each returns a Status and fills err on failure
int setup_validate_mesh(Setup& s, Error& err);
int setup_pairing(Setup& s, Error& err);
int setup_operators(Setup& s, Error& err);
int setup_grid(Setup& s, Error& err);
int setup_spectrum(Setup& s, Error& err);
int setup_precorrection(Setup& s, Error& err);
int setup_near_elements(Setup& s, Error& err);
int run_setup(Setup& s, Error& err);

// Near-element correction, as planned on the host: the sorted near placements of every row
// and, for every vertex of a placement, its output slot (adjacency position, or nnz + the
// index of an extra column); extra columns per row sorted.
struct NearPlan {
  std::vector<int64_t> pptr;   // Np + 1
  std::vector<int64_t> elem;   // tet index, or T + boundary-triangle index
  std::vector<int32_t> img;    // 3 per placement
  std::vector<int64_t> dest;   // 4 per placement
  std::vector<int64_t> xptr;   // Np + 1
  std::vector<int32_t> xcol;
};

// GPU set-up stages (setup_gpu.cu), FP64 on the current device; each fills what its host
// counterpart fills
int spectrum_gpu(Setup& s, Error& err);                                             // s.ghat
int near_eval_gpu(const Setup& s, const NearPlan& plan, std::vector<double>& out, Error& err);
int precorrection_gpu(Setup& s, const std::vector<int32_t>& box, const std::vector<int64_t>& bptr,
                      const std::vector<int32_t>& bl, const std::vector<double>& T0, int R, Error& err);   // s.C

// periodic Green's function of Eq. 15 (k0 = 0), Ewald-type evaluation: the lattice's
// parameters are built here (host); the evaluation itself is sm::pgf_eval (setup_math.hpp),
// shared with the GPU set-up, which copies params() and kflat() to the device
class PeriodicGreen {
 public:
  PeriodicGreen(const double L[3], double eta_scale = 1.0);
  PeriodicGreen(const PeriodicGreen&) = delete;             // params() points into kflat_
  PeriodicGreen& operator=(const PeriodicGreen&) = delete;
  double operator()(double x, double y, double z) const;  // r not on the lattice
  double reg0() const { return reg0_; }                     // lim (G^p - 1/r)
  int dim() const { return dim_; }
  const sm::PgfParams& params() const { return P_; }
  const std::vector<double>& kflat() const { return kflat_; }   // nk x (kx, ky, kz, coefficient)
 private:
  void fill_params();
  int dim_ = 0;
  int ax_[3] = {0, 1, 2};          // periodic axes first, then the open ones
  double L_[3] = {0, 0, 0};
  bool per_[3] = {false, false, false};
  double eta_ = 0;
  int nimg_[3] = {0, 0, 0};
  std::vector<std::array<double, 4>> kvec_;   // (kx, ky, kz, coefficient)
  std::vector<double> gl_u_, gl_w_;           // Gauss-Legendre on [0, 1]
  double reg0_ = 0;
  sm::PgfParams P_;
  std::vector<double> kflat_;
};

// exact potential integrals (Sec. 3.2 near correction)
// int_tri phi_j / |r - r'| dS' for the three hat functions of triangle (a, b, c)
void tri_hat_potentials(const double r[3], const double a[3], const double b[3], const double c[3],
                        double out[3]);
// int_tet dV' / |r - r'|
double tet_potential(const double r[3], const double X[4][3]);

// small thread pool helper: f(begin, end) over [0, n) split in chunks
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f, int64_t min_chunk = 256);

// tetrahedron volume and barycentric gradients
double tet_grads(const double X[4][3], double g[4][3]);

}  // namespace pmfem
